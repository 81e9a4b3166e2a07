"""Python binding of libsbs (include/sbs.h): argument marshalling only.

Every step of the controller runs in the library's CUDA kernels.  PyTorch
provides device memory (through the allocator callbacks below) and streams.
The binding fails loudly when the compiled library is missing; there is no
fallback implementation.

One controller, one warm-started solve per control tick (device inputs)::

    from paper_2403_11383_b300 import sbs, workloads
    cfg = workloads.config("naive_freqset_k10000_h12")   # or a dict of the same keys
    ctl = sbs.Controller(cfg)
    res = ctl.solve(x0, xref, gait, f_ext, shift=1)     # x0 [12], xref [H, 12], f_ext [3] CUDA tensors
    r = sbs.parse_result(res.cpu().numpy())              # u0 (first forces), q_freq, cost_min, status ...

Host inputs: ``ctl.solve_host(...)`` with float32 numpy arrays.  Many
controllers per launch: ``sbs.Batch(n, workspace_bytes).solve(controllers,
[c.problem(...) for c in controllers], results)``.  A request loop with
continuous batching: ``sbs.Server(...).submit(handles, records)`` /
``poll(tickets)``.  Ground-fixed feet pass ``feet=`` ([4, 2] ground positions).

A control loop that solves the same controllers tick after tick packs its
arguments once and edits them in place, so a tick marshals nothing::

    p = ctl.problem(x0, xref, gait, f_ext, shift=1)     # buffers updated in place
    p.gait.phase0 = phase                                # per tick
    ctl.solve_packed(p, res)

    packed = sbs.Packed(controllers, problems)
    packed.problems[i].gait.phase0 = phase_i             # per tick
    batch.solve_packed(packed, results)
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

OK, PENDING = 0, 1
ERR_INVALID_ARG, ERR_OOM, ERR_BUDGET, ERR_CUDA, ERR_TIMEOUT, ERR_DIVERGED = -1, -2, -3, -4, -5, -6
MPPI, ELITE, NAIVE = 0, 1, 2
BUF_MEAN, BUF_VAR, BUF_COST, BUF_FREQ, BUF_ELITE, BUF_MPPI_MEAN = 0, 1, 2, 3, 4, 5
THETA_STORE, THETA_REGENERATE = 0, 1
SPT_NOISE_WARPS = 3  # plain solves: one sample per thread plus a thread drawing its noise one step ahead
MAX_H, MAX_K, MAX_TILE, MAX_FREQ = 128, 1 << 24, 256, 8
BATCH_PERSISTENT, BATCH_GRID = 0, 1


class Model(C.Structure):
    _fields_ = [("mass", C.c_float), ("inertia", C.c_float * 3), ("foot", (C.c_float * 3) * 4),
                ("gravity", C.c_float * 3)]


class Cost(C.Structure):
    _fields_ = [("Q", C.c_float * 12), ("R", C.c_float * 3), ("w_fc", C.c_float), ("mu", C.c_float),
                ("rho", C.c_float), ("f_nominal", C.c_float), ("w_terminal", C.c_float)]


class Config(C.Structure):
    _fields_ = [("K", C.c_int32), ("H", C.c_int32), ("P", C.c_int32), ("method", C.c_int32),
                ("iterations", C.c_int32), ("elite_count", C.c_int32), ("adaptive", C.c_int32),
                ("compare_mppi", C.c_int32), ("dt_us", C.c_uint32), ("q_init", C.c_uint32),
                ("seed", C.c_uint32), ("controller_id", C.c_uint32), ("lam", C.c_float),
                ("f_min", C.c_float), ("f_max", C.c_float), ("sigma_init", C.c_float),
                ("sigma_min", C.c_float), ("sigma_f_init", C.c_float), ("sigma_f_min", C.c_float),
                ("tile", C.c_int32), ("model", Model), ("cost", Cost),
                ("n_freq", C.c_int32), ("freq_set", C.c_uint32 * MAX_FREQ), ("world_feet", C.c_int32),
                ("friction_project", C.c_int32)]


class Gait(C.Structure):
    _fields_ = [("offset", C.c_uint32 * 4), ("duty", C.c_uint32), ("phase0", C.c_uint32)]


class Problem(C.Structure):
    _fields_ = [("x0", C.c_void_p), ("xref", C.c_void_p), ("f_ext", C.c_void_p), ("gait", Gait),
                ("shift", C.c_int32), ("host_memory", C.c_int32), ("feet", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("u0", C.c_float * 12), ("cost_min", C.c_float), ("ess", C.c_float), ("f_mean", C.c_float),
                ("q_freq", C.c_int32), ("status", C.c_int32), ("n_finite", C.c_int32),
                ("iter_lo", C.c_uint32), ("iter_hi", C.c_uint32)]


RESULT_BYTES = C.sizeof(Result)


class ServerConfig(C.Structure):
    _fields_ = [("slots", C.c_int32), ("max_batch", C.c_int32), ("max_pending", C.c_int32), ("plain", C.c_int32),
                ("budget_bytes", C.c_size_t), ("samples_per_thread", C.c_int32), ("theta_mode", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("completed", C.c_uint64), ("ticks", C.c_uint64), ("p50_us", C.c_double), ("p99_us", C.c_double),
                ("max_us", C.c_double), ("mean_us", C.c_double), ("mean_batch", C.c_double),
                ("admission_waits", C.c_uint64), ("max_inflight", C.c_uint64)]


# numpy views of the ABI records, for vectorised marshalling of many requests
PROBLEM_DTYPE = np.dtype([("x0", "<u8"), ("xref", "<u8"), ("f_ext", "<u8"), ("offset", "<u4", (4,)),
                          ("duty", "<u4"), ("phase0", "<u4"), ("shift", "<i4"), ("host_memory", "<i4"),
                          ("feet", "<u8")])
RESULT_DTYPE = np.dtype([("u0", "<f4", (12,)), ("cost_min", "<f4"), ("ess", "<f4"), ("f_mean", "<f4"),
                         ("q_freq", "<i4"), ("status", "<i4"), ("n_finite", "<i4"), ("iter_lo", "<u4"),
                         ("iter_hi", "<u4")])

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class SBSError(RuntimeError):
    def __init__(self, status, what=""):
        super().__init__(f"{what}: {status_str(status)} ({status})")
        self.status = status


_lib = None

# name -> (restype, argtypes); the complete exported ABI of include/sbs.h
ABI = {
    "sbs_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sbs_destroy": (None, [C.c_void_p]),
    "sbs_dim": (C.c_int, [C.c_void_p]),
    "sbs_prepare": (C.c_int, [C.c_void_p]),
    "sbs_device_bytes": (C.c_size_t, [C.c_void_p]),
    "sbs_workspace_bytes": (C.c_size_t, [C.c_void_p]),
    "sbs_workspace_bytes_mode": (C.c_size_t, [C.c_void_p, C.c_int]),
    "sbs_reset": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p]),
    "sbs_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sbs_read": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p]),
    "sbs_state_size": (C.c_size_t, [C.c_void_p]),
    "sbs_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "sbs_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    "sbs_batch_create": (C.c_int, [C.c_int, C.c_int, C.c_size_t, C.c_void_p, C.c_void_p]),
    "sbs_batch_destroy": (None, [C.c_void_p]),
    "sbs_batch_solve": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sbs_batch_solve_host": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sbs_batch_host_inputs": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "sbs_status_str": (C.c_char_p, [C.c_int]),
    "sbs_solve_mppi_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p,
                                        C.c_void_p]),
    "sbs_batch_set_profiling": (C.c_int, [C.c_void_p, C.c_int]),
    "sbs_batch_set_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "sbs_server_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sbs_server_destroy": (None, [C.c_void_p]),
    "sbs_server_submit": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sbs_server_poll": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sbs_server_stats_get": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "sbs_batch_get_mode": (C.c_int, [C.c_void_p]),
    "sbs_batch_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                     C.c_void_p]),
    "sbs_batch_stage_ms": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sbs_batch_set_samples_per_thread": (C.c_int, [C.c_void_p, C.c_int]),
    "sbs_batch_get_samples_per_thread": (C.c_int, [C.c_void_p]),
    "sbs_set_samples_per_thread": (C.c_int, [C.c_void_p, C.c_int]),
    "sbs_set_theta_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "sbs_get_theta_mode": (C.c_int, [C.c_void_p]),
    "sbs_get_samples_per_thread": (C.c_int, [C.c_void_p]),
    "sbs_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "sbs_batch_set_theta_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "sbs_batch_get_theta_mode": (C.c_int, [C.c_void_p]),
    "sbs_shard_exchange_bytes": (C.c_size_t, [C.c_void_p]),
    "sbs_shard_tiles": (C.c_int, [C.c_void_p]),
    "sbs_shard_range": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "sbs_shard_rollout": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "sbs_shard_update": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sbs_fp32_peak": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sbs_sincos": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "sbs_philox4x32_10": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "sbs_sqrt_hw": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "sbs_normals": (C.c_int, [C.c_uint32, C.c_uint32, C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_void_p,
                              C.c_void_p]),
}


def lib_path() -> str:
    """The in-tree library, or the one named by SBS_LIB (an alternative build)."""
    return os.environ.get("SBS_LIB") or _build.LIB


def lib():
    """Load libsbs.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libsbs.so not built ({path}); run `python -m paper_2403_11383_b300.build`")
        L = C.CDLL(path)
        for name, (res, args) in ABI.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_str(s: int) -> str:
    return lib().sbs_status_str(s).decode()


def check(status: int, what: str = "sbs"):
    if status != OK:
        raise SBSError(status, what)


# ----------------------------------------------------------------------------- marshalling

def make_config(cfg: dict, tile: int = 0) -> Config:
    """Config from a workload dict (see workloads.py)."""
    c = Config()
    c.K, c.H, c.P = cfg["K"], cfg["H"], cfg.get("P", 0)
    c.method = {"mppi": MPPI, "elite": ELITE, "naive": NAIVE}[cfg["method"]]
    c.iterations = cfg.get("iterations", 1)
    c.elite_count = cfg.get("elite_count", 1)
    c.adaptive = 1 if cfg.get("adaptive") else 0
    c.compare_mppi = 1 if cfg.get("compare_mppi") else 0
    c.dt_us, c.q_init = cfg["dt_us"], cfg["q_init"]
    c.seed, c.controller_id = cfg["seed"], cfg.get("ctrl", 0)
    c.lam = cfg["lam"]
    c.f_min, c.f_max = cfg["f_min"], cfg["f_max"]
    c.sigma_init, c.sigma_min = cfg["sigma_init"], cfg["sigma_min"]
    c.sigma_f_init, c.sigma_f_min = cfg["sigma_f_init"], cfg["sigma_f_min"]
    c.tile = tile or cfg.get("tile", 0)
    m = cfg["model"]
    c.model.mass = m["mass"]
    c.model.inertia[:] = list(m["inertia"])
    for i in range(4):
        c.model.foot[i][:] = list(m["foot"][i])
    c.model.gravity[:] = list(m["gravity"])
    k = cfg["cost"]
    c.cost.Q[:] = list(k["Q"])
    c.cost.R[:] = list(k["R"])
    c.cost.w_fc, c.cost.mu, c.cost.rho, c.cost.f_nominal = k["w_fc"], k["mu"], k["rho"], k["f_nominal"]
    c.cost.w_terminal = k.get("w_terminal", 0.0)
    fs = list(cfg.get("freq_set_mhz", ()))
    c.n_freq = len(fs)
    for i, f in enumerate(fs[:MAX_FREQ]):
        c.freq_set[i] = f
    c.world_feet = 1 if cfg.get("world_feet") else 0
    c.friction_project = 1 if cfg.get("friction_project") else 0
    return c


def make_gait(g: dict) -> Gait:
    out = Gait()
    out.offset[:] = list(g["offset"])
    out.duty, out.phase0 = g["duty"], g["phase0"]
    return out


def parse_result(buf) -> dict:
    """Decode one sbs_result from bytes / a uint8 array of RESULT_BYTES."""
    raw = bytes(buf) if isinstance(buf, (bytes, bytearray, memoryview)) else np.asarray(buf, dtype=np.uint8).tobytes()
    r = Result.from_buffer_copy(raw[:RESULT_BYTES])
    return {"u0": np.array(r.u0[:], dtype=np.float32), "cost_min": r.cost_min, "ess": r.ess,
            "f_mean": r.f_mean, "q_freq": r.q_freq, "status": r.status, "n_finite": r.n_finite,
            "iter": r.iter_lo | (r.iter_hi << 32)}


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self):
        self._live = {}
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = Allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, ctx):
        import torch
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        except RuntimeError:
            return None
        p = t.data_ptr()
        self._live[p] = t
        return p

    def _do_free(self, ptr, ctx):
        self._live.pop(ptr, None)


_TORCH_ALLOC = None


def torch_allocator() -> TorchAllocator:
    global _TORCH_ALLOC
    if _TORCH_ALLOC is None:
        _TORCH_ALLOC = TorchAllocator()
    return _TORCH_ALLOC


class Controller:
    """One controller instance (sbs_create ... sbs_destroy)."""

    def __init__(self, cfg: dict, tile: int = 0, use_torch_allocator: bool = True):
        self.cfg = cfg
        self._c = make_config(cfg, tile)
        self._h = C.c_void_p()
        alloc = C.byref(torch_allocator().struct) if use_torch_allocator else None
        check(lib().sbs_create(C.byref(self._c), alloc, C.byref(self._h)), "sbs_create")
        self.D = lib().sbs_dim(self._h)
        self.K, self.H = cfg["K"], cfg["H"]

    @property
    def handle(self):
        return self._h

    @property
    def tile(self) -> int:
        """Samples per tile (sbs_config.tile; 0 there selects 128)."""
        return self._c.tile or 128

    def device_bytes(self) -> int:
        return lib().sbs_device_bytes(self._h)

    def set_samples_per_thread(self, spt: int):
        """1, 2, or 0 (default, one): samples each rollout thread of a plain solve
        carries (same results)."""
        check(lib().sbs_set_samples_per_thread(self._h, spt), "sbs_set_samples_per_thread")

    def set_theta_mode(self, mode: int):
        """THETA_STORE or THETA_REGENERATE for plain solves (same results)."""
        check(lib().sbs_set_theta_mode(self._h, mode), "sbs_set_theta_mode")

    def theta_mode(self) -> int:
        return lib().sbs_get_theta_mode(self._h)

    def samples_per_thread(self) -> int:
        return lib().sbs_get_samples_per_thread(self._h)

    def autotune(self, problem: "Problem", result, ticks: int = 5, stream=None):
        """sbs_autotune: time the plain-solve settings on this problem (real
        solves), keep the fastest; returns {(spt, theta_mode): ms}."""
        ms = (C.c_float * 6)()
        ptr = result.data_ptr() if hasattr(result, "data_ptr") else C.addressof(result)
        check(lib().sbs_autotune(self._h, C.byref(problem), C.c_void_p(ptr), ticks, ms, _stream_ptr(stream)),
              "sbs_autotune")
        return {(1 + i // 2, i % 2): ms[i] for i in range(6) if ms[i] >= 0}

    def prepare(self):
        """Allocate the plain-solve workspace now."""
        check(lib().sbs_prepare(self._h), "sbs_prepare")

    def workspace_bytes(self) -> int:
        return lib().sbs_workspace_bytes(self._h)

    def workspace_bytes_mode(self, theta_mode: int) -> int:
        """Batch workspace of one solve in the given deviation mode."""
        return lib().sbs_workspace_bytes_mode(self._h, theta_mode)

    def close(self):
        if self._h:
            lib().sbs_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, gait: dict, it: int = 0, stream=None):
        g = make_gait(gait)
        check(lib().sbs_reset(self._h, C.byref(g), it, _stream_ptr(stream)), "sbs_reset")

    def problem(self, x0, xref, gait, f_ext=None, shift=0, host=False, feet=None) -> Problem:
        p = Problem()
        if feet is not None:
            p.feet = feet.data_ptr() if hasattr(feet, "data_ptr") else feet.ctypes.data
        p.x0 = x0.data_ptr() if hasattr(x0, "data_ptr") else x0.ctypes.data
        p.xref = xref.data_ptr() if hasattr(xref, "data_ptr") else xref.ctypes.data
        if f_ext is None:
            p.f_ext = None
        else:
            p.f_ext = f_ext.data_ptr() if hasattr(f_ext, "data_ptr") else f_ext.ctypes.data
        p.gait = make_gait(gait)
        p.shift = shift
        p.host_memory = 1 if host else 0
        return p

    def solve(self, x0, xref, gait, f_ext=None, shift=0, result=None, stream=None, feet=None):
        """Device solve: x0 [12], xref [H,12], f_ext [3] (and feet [4,2] for world-fixed
        feet) float32 CUDA tensors.  Returns the device result buffer (uint8 tensor of
        RESULT_BYTES)."""
        import torch
        if result is None:
            result = torch.empty(RESULT_BYTES, dtype=torch.uint8, device="cuda")
        p = self.problem(x0, xref, gait, f_ext, shift, host=False, feet=feet)
        check(lib().sbs_solve(self._h, C.byref(p), C.c_void_p(result.data_ptr()), _stream_ptr(stream)),
              "sbs_solve")
        return result

    def solve_host(self, x0, xref, gait, f_ext=None, shift=0, result: Optional[Result] = None, stream=None,
                   feet=None):
        """Host-memory solve: numpy/pinned-CPU float32 inputs; the result struct is
        written on the stream (synchronize before reading)."""
        if result is None:
            result = Result()
        p = self.problem(x0, xref, gait, f_ext, shift, host=True, feet=feet)
        check(lib().sbs_solve(self._h, C.byref(p), C.byref(result), _stream_ptr(stream)), "sbs_solve")
        return result

    def solve_packed(self, problem: Problem, result, stream=None):
        """One solve of a Problem built once by problem() (device or host memory, as
        it says) and edited in place between ticks (problem.gait.phase0,
        problem.shift): nothing is marshalled per call.  result: a uint8 CUDA
        tensor of RESULT_BYTES for device problems, a Result for host problems."""
        out = C.byref(result) if isinstance(result, Result) else C.c_void_p(result.data_ptr())
        check(lib().sbs_solve(self._h, C.byref(problem), out, _stream_ptr(stream)), "sbs_solve")
        return result

    # ---- sample sharding (the exchange between ranks is the caller's; see sharding.py)
    def shard_exchange_bytes(self) -> int:
        return lib().sbs_shard_exchange_bytes(self._h)

    def shard_tiles(self) -> int:
        return lib().sbs_shard_tiles(self._h)

    def shard_rollout(self, problem: Problem, rank: int, world: int, xbuf, stream=None):
        """This rank's tiles of one iteration into xbuf (a CUDA tensor of
        shard_exchange_bytes() bytes), for a device Problem from problem()."""
        check(lib().sbs_shard_rollout(self._h, C.byref(problem), rank, world, C.c_void_p(xbuf.data_ptr()),
                                      _stream_ptr(stream)), "sbs_shard_rollout")

    def shard_update(self, xbuf, result, stream=None):
        """The iteration's update from the exchange buffer summed over ranks;
        result: a uint8 CUDA tensor of RESULT_BYTES."""
        check(lib().sbs_shard_update(self._h, C.c_void_p(xbuf.data_ptr()), C.c_void_p(result.data_ptr()),
                                     _stream_ptr(stream)), "sbs_shard_update")
        return result

    def read(self, which: int, stream=None):
        import torch
        naive_n = max(1, len(self.cfg.get("freq_set_mhz", ()))) + 1  # per-block winners, best block
        n = {BUF_MEAN: self.D, BUF_VAR: self.D, BUF_COST: self.K, BUF_FREQ: self.K,
             BUF_ELITE: self.cfg.get("elite_count", 1) if self.cfg["method"] == "elite" else naive_n,
             BUF_MPPI_MEAN: self.D}[which]
        dt = torch.int32 if which in (BUF_FREQ, BUF_ELITE) else torch.float32
        out = torch.empty(n, dtype=dt, device="cuda")
        check(lib().sbs_read(self._h, which, C.c_void_p(out.data_ptr()), out.numel() * 4, 0, _stream_ptr(stream)),
              "sbs_read")
        return out

    def get_state(self, stream=None) -> bytes:
        n = lib().sbs_state_size(self._h)
        buf = (C.c_uint8 * n)()
        check(lib().sbs_get_state(self._h, buf, n, _stream_ptr(stream)), "sbs_get_state")
        return bytes(buf)

    def set_state(self, blob: bytes, stream=None):
        buf = (C.c_uint8 * len(blob)).from_buffer_copy(blob)
        check(lib().sbs_set_state(self._h, buf, len(blob), _stream_ptr(stream)), "sbs_set_state")


class Batch:
    """Many controllers per persistent, graph-captured launch (sbs_batch_*)."""

    def __init__(self, max_instances: int, workspace_bytes: int, inflight: int = 1, use_torch_allocator: bool = True):
        """workspace_bytes: total scratch budget, split between `inflight` ticks."""
        self._b = C.c_void_p()
        alloc = C.byref(torch_allocator().struct) if use_torch_allocator else None
        check(lib().sbs_batch_create(max_instances, inflight, workspace_bytes, alloc, C.byref(self._b)),
              "sbs_batch_create")

    def close(self):
        if self._b:
            lib().sbs_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mode(self, mode: int):
        check(lib().sbs_batch_set_mode(self._b, mode), "sbs_batch_set_mode")

    def mode(self) -> int:
        return lib().sbs_batch_get_mode(self._b)

    def autotune(self, controllers, problems, results, ticks=5, stream=None):
        """Measure both launch modes on these controllers (real solves) and keep
        the faster; returns (grid_ms, persistent_ms) per tick."""
        n = len(controllers)
        hs = (C.c_void_p * n)(*[c.handle.value for c in controllers])
        ps = (Problem * n)(*problems)
        ms = (C.c_float * 2)()
        check(lib().sbs_batch_autotune(self._b, n, hs, ps, C.c_void_p(results.data_ptr()), ticks, ms,
                                       _stream_ptr(stream)), "sbs_batch_autotune")
        return ms[0], ms[1]

    def set_profiling(self, on: bool):
        check(lib().sbs_batch_set_profiling(self._b, 1 if on else 0), "sbs_batch_set_profiling")

    def set_samples_per_thread(self, spt: int):
        """1, 2, or 0 (default, one): samples each rollout thread carries (same results)."""
        check(lib().sbs_batch_set_samples_per_thread(self._b, spt), "sbs_batch_set_samples_per_thread")

    def samples_per_thread(self) -> int:
        return lib().sbs_batch_get_samples_per_thread(self._b)

    def set_theta_mode(self, mode: int):
        """THETA_STORE or THETA_REGENERATE for the sampled deviations (same results)."""
        check(lib().sbs_batch_set_theta_mode(self._b, mode), "sbs_batch_set_theta_mode")

    def theta_mode(self) -> int:
        return lib().sbs_batch_get_theta_mode(self._b)

    def stage_ms(self):
        """(rollout, selection, refit) milliseconds of the last profiled tick."""
        ms = (C.c_float * 3)()
        check(lib().sbs_batch_stage_ms(self._b, ms), "sbs_batch_stage_ms")
        return list(ms)

    def solve(self, controllers, problems, results, stream=None):
        """controllers: list of Controller; problems: list of Problem (device
        memory); results: uint8 CUDA tensor of n * RESULT_BYTES.  Packs both lists
        on every call; a control loop that solves the same controllers tick after
        tick packs them once (Packed) and calls solve_packed."""
        self.solve_packed(Packed(controllers, problems), results, stream)

    def solve_packed(self, packed: "Packed", results, stream=None):
        """One tick of the packed controllers (no per-call marshalling)."""
        check(lib().sbs_batch_solve(self._b, packed.n, packed.handles, packed.problems,
                                    C.c_void_p(results.data_ptr()), _stream_ptr(stream)), "sbs_batch_solve")


    def solve_host(self, packed: "Packed", results, stream=None):
        """One tick from host memory, end to end (sbs_batch_solve_host): the packed
        problems point at host arrays (host=True), results is a host buffer of
        n * RESULT_BYTES (a ctypes array of Result, or a uint8 numpy array or CPU
        tensor); on return the results are in it."""
        ptr = results.data_ptr() if hasattr(results, "data_ptr") else (
            results.ctypes.data if hasattr(results, "ctypes") else C.addressof(results))
        check(lib().sbs_batch_solve_host(self._b, packed.n, packed.handles, packed.problems, C.c_void_p(ptr),
                                         _stream_ptr(stream)), "sbs_batch_solve_host")

    def host_inputs(self, controllers, gaits, shift=1, with_fext=True):
        """sbs_batch_host_inputs: host problems whose inputs live in the batch's
        pinned staging buffer, packed for solve_host, and one dict of numpy views
        per controller (x0 [12], xref [H, 12], f_ext [3] or None, feet [4, 2] or
        None) to write that controller's inputs into; a solve_host of this Packed
        then copies no input on the host."""
        n = len(controllers)
        hs = (C.c_void_p * n)(*[c.handle.value for c in controllers])
        ps = (Problem * n)()
        check(lib().sbs_batch_host_inputs(self._b, n, hs, 1 if with_fext else 0, ps), "sbs_batch_host_inputs")

        def view(ptr, shape):
            if not ptr:
                return None
            count = int(np.prod(shape))
            return np.ctypeslib.as_array((C.c_float * count).from_address(ptr)).reshape(shape)
        views = []
        for i, c in enumerate(controllers):
            ps[i].gait = make_gait(gaits[i])
            ps[i].shift = shift
            views.append({"x0": view(ps[i].x0, (12,)), "xref": view(ps[i].xref, (c.H, 12)),
                          "f_ext": view(ps[i].f_ext, (3,)), "feet": view(ps[i].feet, (4, 2))})
        return Packed(controllers, list(ps)), views


class Packed:
    """The controller handles and problems of one batch, packed once into the C
    arrays that sbs_batch_solve takes.  A control loop keeps the object and edits
    its entries in place between ticks (packed.problems[i].gait.phase0,
    packed.problems[i].shift, or new device pointers), so a tick marshals nothing."""

    def __init__(self, controllers, problems):
        if len(controllers) != len(problems) or not controllers:
            raise ValueError("one problem per controller, at least one controller")
        self.n = len(controllers)
        self.controllers = list(controllers)  # keeps the handles alive
        self.handles = (C.c_void_p * self.n)(*[c.handle.value for c in controllers])
        self.problems = (Problem * self.n)(*problems)


STATIC_SCRATCH_BYTES = 64 << 20


def solve_mppi_static(cfg: dict, x0, xref, gait, f_ext, shift, state_in, state_out, it, result, stream=None,
                      tile: int = 0):
    """sbs_solve_mppi_static: one MPPI iteration with the library's static scratch
    (no device allocation).  All tensors are CUDA tensors; state_* hold
    [mean | variance]; result is a uint8 tensor of RESULT_BYTES."""
    c = make_config(cfg, tile)
    p = Problem()
    p.x0, p.xref = x0.data_ptr(), xref.data_ptr()
    p.f_ext = None if f_ext is None else f_ext.data_ptr()
    p.gait = make_gait(gait)
    p.shift, p.host_memory = shift, 0
    check(lib().sbs_solve_mppi_static(C.byref(c), C.byref(p), C.c_void_p(state_in.data_ptr()),
                                      C.c_void_p(state_out.data_ptr()), it, C.c_void_p(result.data_ptr()),
                                      _stream_ptr(stream)), "sbs_solve_mppi_static")


def shard_range(ntiles: int, rank: int, world: int):
    """Tiles [begin, end) of rank `rank` of `world` (host arithmetic, no GPU)."""
    b, e = C.c_int(), C.c_int()
    check(lib().sbs_shard_range(ntiles, rank, world, C.byref(b), C.byref(e)), "sbs_shard_range")
    return b.value, e.value


def philox(ctr, key, stream=None):
    """Philox4x32-10 on the device: ctr (n, 4), key (n, 2) int32 CUDA tensors -> (n, 4)."""
    import torch
    n = ctr.shape[0]
    out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    check(lib().sbs_philox4x32_10(C.c_void_p(ctr.data_ptr()), C.c_void_p(key.data_ptr()),
                                  C.c_void_p(out.data_ptr()), n, _stream_ptr(stream)), "sbs_philox4x32_10")
    return out


def sincos(x, stream=None):
    """The model step's attitude sine and cosine of a float32 CUDA tensor:
    returns (sin, cos, sin_packed, cos_packed, sin_library, cos_library,
    sin_hardware, cos_hardware)."""
    import torch
    n = x.numel()
    out = torch.empty(8 * n, dtype=torch.float32, device=x.device)
    check(lib().sbs_sincos(C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), n, _stream_ptr(stream)),
          "sbs_sincos")
    return tuple(out[i * n:(i + 1) * n] for i in range(8))


def sqrt_hw(x, stream=None):
    """The rollout's hardware square root of a float32 CUDA tensor."""
    import torch
    out = torch.empty_like(x)
    check(lib().sbs_sqrt_hw(C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), x.numel(), _stream_ptr(stream)),
          "sbs_sqrt_hw")
    return out


def normals(seed, ctrl, it, k0, nk, nn, stream=None):
    """The controller's normals (frequency, then nn force normals) for nk samples."""
    import torch
    out = torch.empty((nk, nn + 1), dtype=torch.float32, device="cuda")
    check(lib().sbs_normals(seed, ctrl, it, k0, nk, nn, C.c_void_p(out.data_ptr()), _stream_ptr(stream)),
          "sbs_normals")
    return out


class Server:
    """The request loop with continuous batching (sbs_server_*)."""

    def __init__(self, slots=2, max_batch=2048, max_pending=1 << 16, budget_bytes=8 << 30, plain=False,
                 use_torch_allocator=False, samples_per_thread=0, theta_mode=THETA_STORE):
        self._s = C.c_void_p()
        cfg = ServerConfig(slots, max_batch, max_pending, 1 if plain else 0, budget_bytes, samples_per_thread,
                           theta_mode)
        alloc = C.byref(torch_allocator().struct) if use_torch_allocator else None
        check(lib().sbs_server_create(C.byref(cfg), alloc, C.byref(self._s)), "sbs_server_create")

    def close(self):
        if self._s:
            lib().sbs_server_destroy(self._s)
            self._s = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, handles: np.ndarray, problems: np.ndarray) -> np.ndarray:
        """handles: uint64 array of controller handles; problems: PROBLEM_DTYPE
        records with host pointers.  Returns the tickets (uint64)."""
        n = len(handles)
        tickets = np.zeros(n, dtype=np.uint64)
        if n == 0:
            return tickets
        h = np.ascontiguousarray(handles, dtype=np.uint64)
        p = np.ascontiguousarray(problems, dtype=PROBLEM_DTYPE)
        st = lib().sbs_server_submit(self._s, n, h.ctypes.data, p.ctypes.data, tickets.ctypes.data)
        if st == PENDING:
            raise SBSError(st, "sbs_server_submit: queue full")
        check(st, "sbs_server_submit")
        return tickets

    def poll(self, tickets: np.ndarray):
        """Returns (status int32 array, RESULT_DTYPE array)."""
        n = len(tickets)
        status = np.zeros(n, dtype=np.int32)
        res = np.zeros(n, dtype=RESULT_DTYPE)
        if n:
            t = np.ascontiguousarray(tickets, dtype=np.uint64)
            check(lib().sbs_server_poll(self._s, n, t.ctypes.data, res.ctypes.data, status.ctypes.data),
                  "sbs_server_poll")
        return status, res

    def stats(self, reset=False) -> dict:
        st = ServerStats()
        check(lib().sbs_server_stats_get(self._s, C.byref(st), 1 if reset else 0), "sbs_server_stats_get")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}


def fp32_peak(stream=None) -> float:
    f = C.c_double()
    check(lib().sbs_fp32_peak(C.byref(f), _stream_ptr(stream)), "sbs_fp32_peak")
    return f.value
