"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only the test suite, `__graft_entry__.smoke()` and the CPU-baseline leg of the
benchmark may import this package.  It is independent of the CUDA library: it
loads `oracle/_build/libsbs_oracle.so`, built from `sbs_oracle.c` by gcc.

Each wrapper names the paper passage its C function follows (section,
equation or algorithm of Turrisi et al., IROS 2024).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

MPPI, ELITE, NAIVE = 0, 1, 2
OK, DIVERGED = 0, -6
PHASE_ONE = 1_000_000_000
MAX_FREQ = 8


class Params(C.Structure):
    _fields_ = [
        ("K", C.c_int32), ("H", C.c_int32), ("P", C.c_int32),
        ("method", C.c_int32), ("iterations", C.c_int32), ("elite_count", C.c_int32),
        ("adaptive", C.c_int32), ("dt_us", C.c_uint32), ("q_init", C.c_uint32),
        ("seed", C.c_uint32), ("ctrl", C.c_uint32),
        ("lam", C.c_double),
        ("mass", C.c_double), ("inertia", C.c_double * 3), ("foot", C.c_double * 12),
        ("gravity", C.c_double * 3),
        ("Q", C.c_double * 12), ("R", C.c_double * 3), ("w_fc", C.c_double), ("mu", C.c_double),
        ("rho", C.c_double), ("f_nominal", C.c_double),
        ("f_min", C.c_double), ("f_max", C.c_double),
        ("sigma_init", C.c_double), ("sigma_min", C.c_double),
        ("sigma_f_init", C.c_double), ("sigma_f_min", C.c_double),
        ("n_freq", C.c_int32), ("freq_set", C.c_uint32 * MAX_FREQ),
        ("feet_mode", C.c_int32), ("friction_project", C.c_int32),
        ("w_terminal", C.c_double),
    ]


class Gait(C.Structure):
    _fields_ = [("offset", C.c_uint32 * 4), ("duty", C.c_uint32), ("phase0", C.c_uint32)]


_lib = None
_lib_flops = None


def lib():
    global _lib
    if _lib is None:
        _lib = _load(_build.build())
    return _lib


def lib_flops():
    """The FLOP-counting build of the same source (single-threaded)."""
    global _lib_flops
    if _lib_flops is None:
        L = _load(_build.build_flops())
        L.orc_flops_reset.restype = None
        L.orc_flops_reset.argtypes = []
        L.orc_flops_read.restype = None
        L.orc_flops_read.argtypes = [C.c_void_p]
        _lib_flops = L
    return _lib_flops


def _load(path):
    L = C.CDLL(path)
    d, u32, i32, u64, i64, vp = C.c_double, C.c_uint32, C.c_int32, C.c_uint64, C.c_int64, C.c_void_p
    sig = {
        "orc_philox4x32_10": (None, [vp, vp, vp]),
        "orc_box_muller": (None, [u32, u32, vp, vp]),
        "orc_box_muller21": (None, [u32, u32, vp, vp]),
        "orc_uniforms21": (None, [vp, vp]),
        "orc_normal": (d, [u32, u32, u32, u32, u64]),
        "orc_freq_normal": (d, [u32, u32, u32, u64]),
        "orc_normals6": (None, [u32, u32, u32, u32, u64, vp]),
        "orc_quantise_freq": (u32, [d, d, d, d, d, vp]),
        "orc_stance": (C.c_int, [vp, C.c_int, u32, u32, C.c_int]),
        "orc_rotation": (None, [vp, vp]),
        "orc_euler_rates": (None, [vp, vp, vp]),
        "orc_srbd_deriv": (None, [vp, vp, vp, vp, vp]),
        "orc_srbd_step": (None, [vp, vp, vp, vp, d, vp]),
        "orc_srbd_deriv_feet": (None, [vp, vp, vp, vp, vp, vp]),
        "orc_foothold": (None, [vp, vp, vp, u32, u32, C.c_int, vp]),
        "orc_cone_project": (None, [d, vp, vp]),
        "orc_stage_cost": (d, [vp, vp, vp, vp, vp]),
        "orc_spline_basis": (None, [C.c_int, C.c_int, d, vp]),
        "orc_spline_at": (d, [C.c_int, C.c_int, d, vp, d]),
        "orc_dim": (C.c_int, [vp]),
        "orc_sample_dim": (C.c_int, [vp]),
        "orc_freq_bin": (C.c_int, [u32, u32, u32, u64, C.c_int]),
        "orc_naive_sets": (C.c_int, [vp, vp, vp, vp, vp, vp]),
        "orc_init_dist": (None, [vp, vp, vp, vp]),
        "orc_warm_shift": (None, [vp, vp, C.c_int, vp, vp]),
        "orc_rollout": (None, [vp, vp, vp, vp, vp, vp, vp, vp, u64, vp, vp, vp, vp, C.c_int]),
        "orc_rollout_sample": (d, [vp, vp, vp, vp, vp, vp, vp, vp, u64, u32, i64, vp]),
        "orc_mppi": (C.c_int, [vp, vp, C.c_int, C.c_int, d, vp, vp, vp]),
        "orc_elite_select": (None, [vp, C.c_int, C.c_int, vp]),
        "orc_elite_refit": (None, [vp, C.c_int, vp, C.c_int, vp, vp, vp]),
        "orc_first_control": (None, [vp, vp, vp, vp]),
        "orc_solve": (C.c_int, [vp, vp, vp, vp, vp, vp, C.c_int, u64, vp, vp, vp, vp, vp, vp, vp,
                                vp, C.c_int]),
        "orc_max_threads": (C.c_int, []),
        "orc_cost_condition": (d, [vp, vp, vp, vp, vp, vp, vp, vp, u64, u32, d, vp]),
        "orc_cost_condition_all": (None, [vp, vp, vp, vp, vp, vp, vp, vp, u64, d, vp, C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.size, n)
    return a


def make_params(cfg) -> Params:
    """Params from a workload config dict (see paper_2403_11383_b300.workloads)."""
    p = Params()
    p.K, p.H, p.P = cfg["K"], cfg["H"], cfg.get("P", 0)
    p.method = {"mppi": MPPI, "elite": ELITE, "naive": NAIVE}[cfg["method"]]
    p.iterations = cfg.get("iterations", 1)
    p.elite_count = cfg.get("elite_count", 1)
    p.adaptive = 1 if cfg.get("adaptive", False) else 0
    p.dt_us = cfg["dt_us"]
    p.q_init = cfg["q_init"]
    p.seed, p.ctrl = cfg["seed"], cfg.get("ctrl", 0)
    p.lam = cfg["lam"]
    m = cfg["model"]
    p.mass = m["mass"]
    p.inertia[:] = m["inertia"]
    p.foot[:] = list(np.asarray(m["foot"], dtype=np.float64).ravel())
    p.gravity[:] = m["gravity"]
    c = cfg["cost"]
    p.Q[:] = c["Q"]
    p.R[:] = c["R"]
    p.w_fc, p.mu, p.rho, p.f_nominal = c["w_fc"], c["mu"], c["rho"], c["f_nominal"]
    p.f_min, p.f_max = cfg["f_min"], cfg["f_max"]
    p.sigma_init, p.sigma_min = cfg["sigma_init"], cfg["sigma_min"]
    p.sigma_f_init, p.sigma_f_min = cfg["sigma_f_init"], cfg["sigma_f_min"]
    fs = list(cfg.get("freq_set_mhz", []))
    p.n_freq = len(fs)
    for i, f in enumerate(fs):
        p.freq_set[i] = f
    p.feet_mode = 1 if cfg.get("world_feet") else 0
    p.friction_project = 1 if cfg.get("friction_project") else 0
    p.w_terminal = cfg["cost"].get("w_terminal", 0.0)
    return p


def make_gait(g) -> Gait:
    out = Gait()
    out.offset[:] = list(g["offset"])
    out.duty = g["duty"]
    out.phase0 = g["phase0"]
    return out


# ----------------------------------------------------------------------------- primitives

def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def box_muller(x, y):
    z0, z1 = C.c_double(), C.c_double()
    lib().orc_box_muller(x, y, C.byref(z0), C.byref(z1))
    return z0.value, z1.value


def box_muller21(a, b):
    z0, z1 = C.c_double(), C.c_double()
    lib().orc_box_muller21(a, b, C.byref(z0), C.byref(z1))
    return z0.value, z1.value


def uniforms21(words):
    w = np.ascontiguousarray(words, dtype=np.uint32)
    u = np.zeros(6, dtype=np.uint32)
    lib().orc_uniforms21(_p(w), _p(u))
    return u


def normal(seed, ctrl, k, n, it):
    return lib().orc_normal(seed, ctrl, k, n, it)


def normals6(seed, ctrl, k, d, it):
    """The six force normals of draw d >= 1 (one Philox block, three Box-Muller pairs)."""
    out = np.zeros(6)
    lib().orc_normals6(seed, ctrl, k, d, it, _p(out))
    return out


def freq_normal(seed, ctrl, k, it):
    return lib().orc_freq_normal(seed, ctrl, k, it)


def quantise_freq(mu_f, sigma_f, z, f_min, f_max):
    m = C.c_double()
    q = lib().orc_quantise_freq(mu_f, sigma_f, z, f_min, f_max, C.byref(m))
    return q, m.value


def stance(gait, leg, q_mhz, dt_us, j):
    """Contact flag of one leg at step j (Sec. IV-C)."""
    g = make_gait(gait) if isinstance(gait, dict) else gait
    return lib().orc_stance(C.byref(g), leg, q_mhz, dt_us, j)


def rotation(rpy):
    r = _f64(rpy, 3)
    out = np.zeros(9)
    lib().orc_rotation(_p(r), _p(out))
    return out.reshape(3, 3)


def euler_rates(rpy, w):
    r, ww = _f64(rpy, 3), _f64(w, 3)
    out = np.zeros(3)
    lib().orc_euler_rates(_p(r), _p(ww), _p(out))
    return out


def srbd_deriv(params, x, gamma, f_ext=None):
    """Right-hand side of Eq. (1)."""
    xx, gg = _f64(x, 12), _f64(gamma, 12)
    fe = None if f_ext is None else _f64(f_ext, 3)
    out = np.zeros(12)
    lib().orc_srbd_deriv(C.byref(params), _p(xx), _p(gg), _p(fe), _p(out))
    return out


def srbd_deriv_feet(params, x, gamma, feet, f_ext=None):
    """Right-hand side of Eq. (1) with world-fixed contact points (x, y) on the ground."""
    xx, gg, ff = _f64(x, 12), _f64(gamma, 12), _f64(feet, 8)
    fe = None if f_ext is None else _f64(f_ext, 3)
    out = np.zeros(12)
    lib().orc_srbd_deriv_feet(C.byref(params), _p(xx), _p(gg), _p(fe), _p(ff), _p(out))
    return out


def foothold(params, x, vd, q_mhz, duty, leg):
    """Touchdown foothold (x, y) of one leg (Sec. IV-D)."""
    xx, v = _f64(x, 12), _f64(vd, 2)
    out = np.zeros(2)
    lib().orc_foothold(C.byref(params), _p(xx), _p(v), q_mhz, duty, leg, _p(out))
    return out


def cone_project(mu, force):
    """Orthogonal projection of a force onto the friction cone (Sec. IV-B)."""
    f = _f64(force, 3)
    out = np.zeros(3)
    lib().orc_cone_project(mu, _p(f), _p(out))
    return out


def _feet(params, feet):
    if not params.feet_mode:
        return None
    assert feet is not None, "world-fixed feet need the feet's ground positions at t_0"
    return _f64(feet, 8)


def srbd_step(params, x, gamma, dt, f_ext=None):
    xx, gg = _f64(x, 12), _f64(gamma, 12)
    fe = None if f_ext is None else _f64(f_ext, 3)
    out = np.zeros(12)
    lib().orc_srbd_step(C.byref(params), _p(xx), _p(gg), _p(fe), dt, _p(out))
    return out


def stage_cost(params, x, xr, gamma, stance_flags):
    xx, rr, gg = _f64(x, 12), _f64(xr, 12), _f64(gamma, 12)
    st = np.ascontiguousarray(stance_flags, dtype=np.int32)
    return lib().orc_stage_cost(C.byref(params), _p(xx), _p(rr), _p(gg), _p(st))


def spline_basis(H, P, dt):
    """H x P natural-cubic-spline basis (Sec. IV-B)."""
    B = np.zeros((H, P))
    lib().orc_spline_basis(H, P, dt, _p(B))
    return B


def spline_at(H, P, dt, y, t):
    yy = _f64(y, P)
    return lib().orc_spline_at(H, P, dt, _p(yy), t)


def dim(params):
    """Length of the distribution's mean (one force block per set frequency)."""
    return lib().orc_dim(C.byref(params))


def sample_dim(params):
    """Length of one sample's decision vector."""
    return lib().orc_sample_dim(C.byref(params))


def freq_bin(seed, ctrl, k, it, n):
    """Set entry drawn by sample k for a discrete frequency set of n values (Sec. V)."""
    return lib().orc_freq_bin(seed, ctrl, k, it, n)


def naive_sets(params, J, q, theta, mean):
    """Naive update over a discrete frequency set (Alg. 3 per frequency's Gaussian).
    Returns (entry of the best sample or -1, per-entry winners, new mean)."""
    J = _f64(J, params.K)
    q = np.ascontiguousarray(q, dtype=np.uint32)
    theta = _f64(theta)
    mean = _f64(mean, dim(params)).copy()
    best = np.zeros(max(1, params.n_freq), dtype=np.int32)
    bs = lib().orc_naive_sets(C.byref(params), _p(J), _p(q), _p(theta), _p(mean), _p(best))
    return bs, best[:params.n_freq], mean


def init_dist(params, gait):
    D = dim(params)
    mean, var = np.zeros(D), np.zeros(D)
    lib().orc_init_dist(C.byref(params), C.byref(gait), _p(mean), _p(var))
    return mean, var


def warm_shift(params, gait, shift, mean, var):
    mean = _f64(mean).copy()
    var = _f64(var).copy()
    lib().orc_warm_shift(C.byref(params), C.byref(gait), shift, _p(mean), _p(var))
    return mean, var


def rollout(params, gait, x0, xref, f_ext, mean, var, it, want_theta=False, nthreads=1, feet=None):
    """Costs of all K samples of iteration `it` (Alg. 2 for each sample)."""
    K, D = params.K, dim(params)
    ft = _feet(params, feet)
    x0 = _f64(x0, 12)
    xref = _f64(xref, 12 * params.H)
    fe = None if f_ext is None else _f64(f_ext, 3)
    mean, var = _f64(mean, D), _f64(var, D)
    J = np.zeros(K)
    q = np.zeros(K, dtype=np.uint32)
    margin = np.zeros(K)
    theta = np.zeros((K, sample_dim(params))) if want_theta else None
    lib().orc_rollout(C.byref(params), C.byref(gait), _p(x0), _p(xref), _p(fe), _p(ft), _p(mean), _p(var),
                      it, _p(J), _p(q), _p(theta), _p(margin), nthreads)
    return J, q, theta, margin


def rollout_sample(params, gait, x0, xref, f_ext, mean, var, it, k, q_override=-1, feet=None):
    D = dim(params)
    ft = _feet(params, feet)
    x0 = _f64(x0, 12)
    xref = _f64(xref, 12 * params.H)
    fe = None if f_ext is None else _f64(f_ext, 3)
    mean, var = _f64(mean, D), _f64(var, D)
    theta = np.zeros(sample_dim(params))
    J = lib().orc_rollout_sample(C.byref(params), C.byref(gait), _p(x0), _p(xref), _p(fe), _p(ft),
                                 _p(mean), _p(var), it, k, q_override, _p(theta))
    return J, theta


def mppi(J, theta, lam):
    """MPPI UpdateMean (Alg. 5). Returns (status, mean, ess, beta)."""
    J = _f64(J)
    theta = _f64(theta)
    K, D = theta.shape
    mean = np.zeros(D)
    ess, beta = C.c_double(), C.c_double()
    st = lib().orc_mppi(_p(J), _p(theta), K, D, lam, _p(mean), C.byref(ess), C.byref(beta))
    return st, mean, ess.value, beta.value


def elite_select(J, Ke):
    J = _f64(J)
    idx = np.zeros(Ke, dtype=np.int32)
    lib().orc_elite_select(_p(J), J.size, Ke, _p(idx))
    return idx


def elite_refit(theta, idx, var_floor):
    theta = _f64(theta)
    K, D = theta.shape
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    fl = _f64(var_floor, D)
    mean, var = np.zeros(D), np.zeros(D)
    lib().orc_elite_refit(_p(theta), D, _p(idx), idx.size, _p(fl), _p(mean), _p(var))
    return mean, var


def first_control(params, gait, mean):
    u0 = np.zeros(12)
    m = _f64(mean)
    lib().orc_first_control(C.byref(params), C.byref(gait), _p(m), _p(u0))
    return u0


def solve(params, gait, x0, xref, f_ext, shift, iter0, mean, var, nthreads=1, feet=None):
    """One controller solve (Alg. 4, Alg. 1 iterated). Returns a dict."""
    K, D = params.K, dim(params)
    ft = _feet(params, feet)
    mean = _f64(mean, D).copy()
    var = _f64(var, D).copy()
    x0 = _f64(x0, 12)
    xref = _f64(xref, 12 * params.H)
    fe = None if f_ext is None else _f64(f_ext, 3)
    u0 = np.zeros(12)
    info = np.zeros(4)
    J = np.zeros(K)
    q = np.zeros(K, dtype=np.uint32)
    Ke = max(1, params.elite_count, params.n_freq)
    elite = np.full(Ke, -1, dtype=np.int32)
    mppi_mean = np.zeros(D)
    st = lib().orc_solve(C.byref(params), C.byref(gait), _p(x0), _p(xref), _p(fe), _p(ft), shift, iter0,
                         _p(mean), _p(var), _p(u0), _p(info), _p(J), _p(q), _p(elite),
                         _p(mppi_mean), nthreads)
    return {"status": st, "mean": mean, "var": var, "u0": u0, "beta": info[0], "ess": info[1],
            "f_mean": info[2], "J": J, "q": q, "elite": elite, "mppi_mean": mppi_mean}


EPS_FP32 = 2.0 ** -23


def cost_condition(params, gait, x0, xref, f_ext, mean, var, it, k, eps=EPS_FP32, feet=None):
    """Relative change of sample k's cost under rounding-sized perturbations."""
    D = dim(params)
    ft = _feet(params, feet)
    x0 = _f64(x0, 12)
    xref = _f64(xref, 12 * params.H)
    fe = None if f_ext is None else _f64(f_ext, 3)
    mean, var = _f64(mean, D), _f64(var, D)
    J = C.c_double()
    kap = lib().orc_cost_condition(C.byref(params), C.byref(gait), _p(x0), _p(xref), _p(fe), _p(ft), _p(mean),
                                   _p(var), it, k, eps, C.byref(J))
    return kap, J.value


def cost_condition_all(params, gait, x0, xref, f_ext, mean, var, it, eps=EPS_FP32, nthreads=1, feet=None):
    D = dim(params)
    ft = _feet(params, feet)
    x0 = _f64(x0, 12)
    xref = _f64(xref, 12 * params.H)
    fe = None if f_ext is None else _f64(f_ext, 3)
    mean, var = _f64(mean, D), _f64(var, D)
    kap = np.zeros(params.K)
    lib().orc_cost_condition_all(C.byref(params), C.byref(gait), _p(x0), _p(xref), _p(fe), _p(ft), _p(mean),
                                 _p(var), it, eps, _p(kap), nthreads)
    return kap


def max_threads():
    return lib().orc_max_threads()


# ----------------------------------------------------------------------------- FLOP counts

FLOP_KEYS = ("add", "mul", "div", "sqrt", "fn")


def _flops_read():
    out = np.zeros(5, dtype=np.uint64)
    lib_flops().orc_flops_read(_p(out))
    d = dict(zip(FLOP_KEYS, (int(v) for v in out)))
    d["flop"] = d["add"] + d["mul"] + d["div"] + d["sqrt"]
    return d


def count_rollout(params, gait, x0, xref, f_ext, mean, var, it, k=0, feet=None):
    """Floating-point operations of sample k's rollout in the counting build:
    sampling, policy, stage cost and dynamics (Alg. 1 Sampling, Alg. 2), with the
    sample's cost.  The per-solve set-up that orc_rollout_sample also performs
    (the spline basis, and one square root per distribution entry for its
    standard deviation) is counted on its own and subtracted."""
    L = lib_flops()
    D = dim(params)
    ft = _feet(params, feet)
    x0, xref = _f64(x0, 12), _f64(xref, 12 * params.H)
    fe = None if f_ext is None else _f64(f_ext, 3)
    mean, var = _f64(mean, D), _f64(var, D)
    theta = np.zeros(sample_dim(params))
    L.orc_flops_reset()
    J = L.orc_rollout_sample(C.byref(params), C.byref(gait), _p(x0), _p(xref), _p(fe), _p(ft), _p(mean), _p(var),
                             it, k, -1, _p(theta))
    total = _flops_read()
    L.orc_flops_reset()
    if params.P > 0:
        L.orc_spline_basis(params.H, params.P, params.dt_us * 1e-6, _p(np.zeros(params.H * params.P)))
    setup = _flops_read()
    setup["sqrt"] += D
    out = {key: total[key] - setup[key] for key in FLOP_KEYS}
    out["flop"] = out["add"] + out["mul"] + out["div"] + out["sqrt"]
    return out, float(J)


def count_mppi(J, theta, lam):
    """Floating-point operations of the MPPI update (Alg. 5) over K samples."""
    L = lib_flops()
    J, theta = _f64(J), _f64(theta)
    K, D = theta.shape
    mean = np.zeros(D)
    ess, beta = C.c_double(), C.c_double()
    L.orc_flops_reset()
    L.orc_mppi(_p(J), _p(theta), K, D, lam, _p(mean), C.byref(ess), C.byref(beta))
    return _flops_read()
