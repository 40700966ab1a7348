"""ctypes binding of liblbm.so: the same entry points as include/lbm.h.

Only argument marshalling happens here (numpy arrays <-> pointers, status
codes -> LbmError); every step of the update runs in the CUDA library.
"""
import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int64, c_size_t, c_uint8, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA = 0, -1, -2, -3
LBM_ERR_TIMEOUT, LBM_ERR_NONFINITE, LBM_ERR_STATE = -4, -5, -6
LBM_D3Q19_MRT_LES, LBM_D3Q27_FCLB = 0, 1
LBM_F64, LBM_F32, LBM_F16 = 0, 1, 2
LBM_MAX_LEVELS = 4
MODELS = {"d3q19": LBM_D3Q19_MRT_LES, "d3q27": LBM_D3Q27_FCLB}
STORAGES = {"f64": LBM_F64, "f32": LBM_F32, "f16": LBM_F16}
EXPORTED = ["lbm_plan", "lbm_create", "lbm_create_error", "lbm_set_inflow", "lbm_set_outlet",
            "lbm_init_equilibrium",
            "lbm_set_force", "lbm_step", "lbm_sync", "lbm_macroscopic", "lbm_mass_momentum",
            "lbm_get_state", "lbm_set_state", "lbm_get_cells", "lbm_get_step", "lbm_set_step",
            "lbm_set_profiling", "lbm_get_profile", "lbm_get_tuning", "lbm_last_error", "lbm_destroy",
            "lbm_mass_momentum_noalloc", "lbm_adjoint_forward", "lbm_adjoint_backward", "lbm_adjoint_generation",
            "lbm_get_strain", "lbm_set_strain", "lbm_raw_state_bytes", "lbm_get_raw_state",
            "lbm_set_raw_state", "lbm_stats_reset", "lbm_stats_accumulate", "lbm_stats_get",
            "lbm_stats_radial", "lbm_jet_fit",
            "lbm_shard_plan", "lbm_shard_create", "lbm_shard_part", "lbm_shard_halo_bytes", "lbm_shard_set_inflow",
            "lbm_shard_init_equilibrium", "lbm_shard_step", "lbm_shard_sync", "lbm_shard_get_state",
            "lbm_shard_macroscopic", "lbm_shard_mass_momentum", "lbm_shard_last_error", "lbm_shard_destroy"]
NOALLOC_MAX_BLOCKS = 65536


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("lbm status %d: %s" % (status, msg))
        self.status = status


class lbm_grid(ctypes.Structure):
    _fields_ = [("nbx", c_int), ("nby", c_int), ("nbz", c_int), ("periodic_x", c_int),
                ("levels", c_int), ("refine", POINTER(c_uint8)), ("walls", c_int), ("slip", c_int),
                ("outlet", c_int), ("nozzle_y0", c_double), ("nozzle_z0", c_double), ("nozzle_r", c_double),
                ("nozzle_x0", c_double), ("nozzle_x1", c_double)]


class lbm_plan_info(ctypes.Structure):
    _fields_ = [("levels", c_int)] + [
        (n, c_int64 * LBM_MAX_LEVELS) for n in
        ("blocks", "level_blocks", "active_cells", "updated_cells", "hidden_cells", "ghost_cells",
         "bc_cells")] + [("updates_per_coarse_step", c_int64),
                         ("active_updates_per_coarse_step", c_int64), ("device_bytes", c_int64),
                         ("nozzle_level", c_int), ("solid_cells", c_int64), ("nozzle_links", c_int64)]


_lib = None


def load():
    """Load liblbm.so (built by __graft_entry__.build()); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblbm.so not built at %s: run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, D = POINTER, POINTER(c_double)
    sig = {
        "lbm_plan": (c_int, [P(lbm_grid), c_int, c_int, P(lbm_plan_info)]),
        "lbm_create": (c_int, [P(c_void_p), c_int, c_int, P(lbm_grid), c_double, c_double, c_void_p]),
        "lbm_create_error": (c_char_p, []),
        "lbm_set_inflow": (c_int, [c_void_p, c_double, c_double, c_double, c_double, c_double, c_uint64]),
        "lbm_set_outlet": (c_int, [c_void_p, c_double]),
        "lbm_init_equilibrium": (c_int, [c_void_p, c_int, D, D]),
        "lbm_set_force": (c_int, [c_void_p, D]),
        "lbm_step": (c_int, [c_void_p, c_int]),
        "lbm_sync": (c_int, [c_void_p]),
        "lbm_macroscopic": (c_int, [c_void_p, c_int, D, D]),
        "lbm_mass_momentum": (c_int, [c_void_p, D]),
        "lbm_get_state": (c_int, [c_void_p, c_int, D, c_size_t]),
        "lbm_set_state": (c_int, [c_void_p, c_int, D, c_size_t]),
        "lbm_get_cells": (c_int, [c_void_p, c_int, c_size_t, P(c_int64), D]),
        "lbm_get_strain": (c_int, [c_void_p, c_int, D, c_size_t]),
        "lbm_raw_state_bytes": (c_int, [c_void_p, c_int, P(c_size_t)]),
        "lbm_stats_reset": (c_int, [c_void_p]),
        "lbm_stats_accumulate": (c_int, [c_void_p]),
        "lbm_stats_get": (c_int, [c_void_p, c_int, D, D, P(c_int64)]),
        "lbm_stats_radial": (c_int, [c_void_p, c_int, c_double, c_double, c_double, c_int, c_int, D, D, D,
                                     P(c_int64)]),
        "lbm_jet_fit": (c_int, [c_int, c_double, D, D, P(c_int64), D]),
        "lbm_get_raw_state": (c_int, [c_void_p, c_int, c_void_p, c_size_t]),
        "lbm_set_raw_state": (c_int, [c_void_p, c_int, c_void_p, c_size_t]),
        "lbm_set_strain": (c_int, [c_void_p, c_int, D, c_size_t]),
        "lbm_get_step": (c_int, [c_void_p, P(c_int64)]),
        "lbm_set_step": (c_int, [c_void_p, c_int64]),
        "lbm_set_profiling": (c_int, [c_void_p, c_int]),
        "lbm_get_profile": (c_int, [c_void_p, D, P(c_int64)]),
        "lbm_get_tuning": (c_int, [c_void_p, P(c_int), P(c_int), P(c_int)]),
        "lbm_last_error": (c_char_p, [c_void_p]),
        "lbm_destroy": (None, [c_void_p]),
        "lbm_mass_momentum_noalloc": (c_int, [c_int, c_int, c_void_p, c_int64, c_void_p, c_void_p]),
        "lbm_adjoint_forward": (c_int, [c_void_p, c_int, c_int]),
        "lbm_adjoint_backward": (c_int, [c_void_p, D, D]),
        "lbm_adjoint_generation": (c_int, [c_void_p, P(c_uint64), P(c_int)]),
        "lbm_shard_plan": (c_int, [P(lbm_grid), c_int, P(c_int)]),
        "lbm_shard_create": (c_int, [P(c_void_p), c_int, c_int, P(lbm_grid), c_double, c_double, c_int, c_void_p]),
        "lbm_shard_part": (c_int, [c_void_p, c_int, P(c_void_p), P(c_int), P(c_int)]),
        "lbm_shard_halo_bytes": (c_int, [c_void_p, P(c_int64)]),
        "lbm_shard_set_inflow": (c_int, [c_void_p, c_double, c_double, c_double, c_double, c_double, c_uint64]),
        "lbm_shard_init_equilibrium": (c_int, [c_void_p, c_int, D, D]),
        "lbm_shard_step": (c_int, [c_void_p, c_int]),
        "lbm_shard_sync": (c_int, [c_void_p]),
        "lbm_shard_get_state": (c_int, [c_void_p, c_int, D, c_size_t]),
        "lbm_shard_macroscopic": (c_int, [c_void_p, c_int, D, D]),
        "lbm_shard_mass_momentum": (c_int, [c_void_p, D]),
        "lbm_shard_last_error": (c_char_p, [c_void_p]),
        "lbm_shard_destroy": (None, [c_void_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(POINTER(c_double)) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def make_grid(nb, periodic_x=True, refine=(), walls=0, slip=0, outlet=0, nozzle=None):
    """lbm_grid from coarse block counts nb = (nbx, nby, nbz), refine flags
    (list of arrays shaped (nbz*2^l, nby*2^l, nbx*2^l)), the wall faces
    (bit 0/1 low/high y, 2/3 low/high z; slip the free-slip subset), the
    outlet type (0 zero-gradient, 1 fixed pressure) and the nozzle
    (y0, z0, r, x0, x1) or None.  Returns (grid, keepalive)."""
    flags = [np.ascontiguousarray(np.asarray(r, dtype=np.uint8)).reshape(-1) for r in refine]
    buf = np.concatenate(flags) if flags else np.zeros(1, dtype=np.uint8)
    g = lbm_grid(int(nb[0]), int(nb[1]), int(nb[2]), 1 if periodic_x else 0, len(flags) + 1,
                 buf.ctypes.data_as(POINTER(c_uint8)), int(walls), int(slip), int(outlet),
                 *(float(v) for v in (nozzle if nozzle is not None else (0, 0, 0, 0, 0))))
    return g, buf


def lbm_plan(nb, periodic_x=True, refine=(), model="d3q19", storage="f32", walls=0, slip=0, outlet=0,
             nozzle=None):
    lib = load()
    g, keep = make_grid(nb, periodic_x, refine, walls, slip, outlet, nozzle)
    info = lbm_plan_info()
    st = lib.lbm_plan(ctypes.byref(g), MODELS[model], STORAGES[storage], ctypes.byref(info))
    if st != LBM_OK:
        raise LbmError(st, "invalid grid")
    return info


class Context:
    """An lbm_ctx handle with the level sizes needed to shape arrays."""

    def __init__(self, handle, model, nb, levels):
        self.h = handle
        self.model = model
        self.Q = 19 if model == "d3q19" else 27
        self.nb = tuple(nb)
        self.levels = levels

    def dims(self, level):
        s = 8 << level
        return (self.nb[0] * s, self.nb[1] * s, self.nb[2] * s)  # NX, NY, NZ

    def ncells(self, level):
        NX, NY, NZ = self.dims(level)
        return NX * NY * NZ


def _check(ctx, st):
    if st != LBM_OK:
        msg = load().lbm_last_error(ctx.h if ctx is not None else None)
        raise LbmError(st, msg.decode() if msg else "")


def lbm_create(model, storage, nb, periodic_x=True, refine=(), omega=1.0, cs=0.0, stream=None,
               walls=0, slip=0, outlet=0, nozzle=None):
    lib = load()
    g, keep = make_grid(nb, periodic_x, refine, walls, slip, outlet, nozzle)
    h = c_void_p()
    st = lib.lbm_create(ctypes.byref(h), MODELS[model], STORAGES[storage], ctypes.byref(g),
                        float(omega), float(cs), stream)
    if st != LBM_OK:
        raise LbmError(st, lib.lbm_create_error().decode())
    return Context(h, model, nb, g.levels)


def lbm_destroy(ctx):
    if ctx is not None and ctx.h:
        load().lbm_destroy(ctx.h)
        ctx.h = None


def lbm_set_inflow(ctx, y0, z0, diameter, u_in, perturb=0.01, seed=0):
    _check(ctx, load().lbm_set_inflow(ctx.h, y0, z0, diameter, u_in, perturb, int(seed)))


def lbm_set_outlet(ctx, rho_out):
    _check(ctx, load().lbm_set_outlet(ctx.h, float(rho_out)))


def lbm_init_equilibrium(ctx, level, rho=None, u=None):
    r, v = _f64(rho), _f64(u)
    _check(ctx, load().lbm_init_equilibrium(ctx.h, level, _dptr(r), _dptr(v)))


def lbm_set_force(ctx, F):
    a = _f64(F)
    _check(ctx, load().lbm_set_force(ctx.h, _dptr(a)))


def lbm_step(ctx, n=1):
    _check(ctx, load().lbm_step(ctx.h, int(n)))


def lbm_sync(ctx):
    _check(ctx, load().lbm_sync(ctx.h))


def lbm_macroscopic(ctx, level):
    NX, NY, NZ = ctx.dims(level)
    rho = np.empty((NZ, NY, NX))
    u = np.empty((3, NZ, NY, NX))
    _check(ctx, load().lbm_macroscopic(ctx.h, level, _dptr(rho), _dptr(u)))
    return rho, u


def lbm_mass_momentum(ctx):
    out = np.empty(4)
    _check(ctx, load().lbm_mass_momentum(ctx.h, _dptr(out)))
    return out


def lbm_get_state(ctx, level):
    NX, NY, NZ = ctx.dims(level)
    f = np.empty((ctx.Q, NZ, NY, NX))
    _check(ctx, load().lbm_get_state(ctx.h, level, _dptr(f), f.size))
    return f


def lbm_set_state(ctx, level, f):
    a = _f64(f)
    _check(ctx, load().lbm_set_state(ctx.h, level, _dptr(a), a.size))


def lbm_stats_reset(ctx):
    _check(ctx, load().lbm_stats_reset(ctx.h))


def lbm_stats_accumulate(ctx):
    _check(ctx, load().lbm_stats_accumulate(ctx.h))


def lbm_stats_get(ctx, level):
    """(mean [4, NZ, NY, NX] of rho, u_x, u_y, u_z; variance [3, NZ, NY, NX]
    of u; number of samples) of the accumulated time statistics."""
    NX, NY, NZ = ctx.dims(level)
    mean = np.empty((4, NZ, NY, NX))
    var = np.empty((3, NZ, NY, NX))
    n = c_int64()
    _check(ctx, load().lbm_stats_get(ctx.h, level, _dptr(mean), _dptr(var), ctypes.byref(n)))
    return mean, var, n.value


def lbm_stats_radial(ctx, level, y0, z0, dr, nbins, x_stations):
    """Ring profiles (mean_ux, var_ux, counts), each [nstations][nbins]."""
    xs = _f64(np.asarray(x_stations, dtype=np.float64).reshape(-1))
    m = np.empty((len(xs), int(nbins)))
    v = np.empty_like(m)
    c = np.empty(m.shape, dtype=np.int64)
    _check(ctx, load().lbm_stats_radial(ctx.h, int(level), float(y0), float(z0), float(dr), int(nbins), len(xs),
                                        _dptr(xs), _dptr(m), _dptr(v), c.ctypes.data_as(POINTER(c_int64))))
    return m, v, c


def lbm_jet_fit(mean_ux, var_ux, counts, dr):
    """(u_m, b_e, tI, a, c) of one station's ring profile."""
    m, v = _f64(mean_ux), _f64(var_ux)
    c = np.ascontiguousarray(counts, dtype=np.int64)
    out = np.empty(5)
    st = load().lbm_jet_fit(len(m), float(dr), _dptr(m), _dptr(v), c.ctypes.data_as(POINTER(c_int64)), _dptr(out))
    if st != LBM_OK:
        raise LbmError(st, "lbm_jet_fit")
    return tuple(float(x) for x in out)


def lbm_raw_state_bytes(ctx, level):
    n = c_size_t()
    _check(ctx, load().lbm_raw_state_bytes(ctx.h, level, ctypes.byref(n)))
    return n.value


def lbm_get_raw_state(ctx, level):
    """The level's device state as stored (bit-exact checkpoint), as uint8."""
    buf = np.empty(lbm_raw_state_bytes(ctx, level), dtype=np.uint8)
    _check(ctx, load().lbm_get_raw_state(ctx.h, level, buf.ctypes.data_as(c_void_p), buf.size))
    return buf


def lbm_set_raw_state(ctx, level, buf):
    b = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(ctx, load().lbm_set_raw_state(ctx.h, level, b.ctypes.data_as(c_void_p), b.size))


def lbm_get_strain(ctx, level):
    NX, NY, NZ = ctx.dims(level)
    S = np.empty((NZ, NY, NX))
    _check(ctx, load().lbm_get_strain(ctx.h, level, _dptr(S), S.size))
    return S


def lbm_set_strain(ctx, level, S):
    a = _f64(S)
    _check(ctx, load().lbm_set_strain(ctx.h, level, _dptr(a), a.size))


def lbm_get_cells(ctx, level, cells):
    c = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.empty((c.size, ctx.Q))
    _check(ctx, load().lbm_get_cells(ctx.h, level, c.size, c.ctypes.data_as(POINTER(c_int64)),
                                     _dptr(out)))
    return out


def lbm_get_step(ctx):
    s = c_int64()
    _check(ctx, load().lbm_get_step(ctx.h, ctypes.byref(s)))
    return s.value


def lbm_set_step(ctx, step):
    _check(ctx, load().lbm_set_step(ctx.h, int(step)))


def lbm_set_profiling(ctx, enable):
    _check(ctx, load().lbm_set_profiling(ctx.h, 1 if enable else 0))


def lbm_get_profile(ctx):
    ms = np.zeros(5)
    n = (c_int64 * 5)()
    _check(ctx, load().lbm_get_profile(ctx.h, _dptr(ms), n))
    return ms, np.array(list(n), dtype=np.int64)


def lbm_adjoint_forward(ctx, T, checkpoint_every):
    _check(ctx, load().lbm_adjoint_forward(ctx.h, int(T), int(checkpoint_every)))


def lbm_adjoint_generation(ctx):
    """(generation, checkpoint_every) of the recorded adjoint forward; (0, 0) if none."""
    g, e = c_uint64(0), c_int(0)
    _check(ctx, load().lbm_adjoint_generation(ctx.h, ctypes.byref(g), ctypes.byref(e)))
    return int(g.value), int(e.value)


def lbm_adjoint_backward(ctx, dLdf_T):
    """dL/dF (3, NZ, NY, NX) from dL/df_T (27, NZ, NY, NX)."""
    NX, NY, NZ = ctx.dims(0)
    g = _f64(dLdf_T)
    out = np.empty((3, NZ, NY, NX))
    _check(ctx, load().lbm_adjoint_backward(ctx.h, _dptr(g), _dptr(out)))
    return out


def lbm_get_tuning(ctx):
    """(threads per CTA, min resident CTAs per SM compiled for, CTAs per launch or 0)."""
    t, m, c = c_int(), c_int(), c_int()
    _check(ctx, load().lbm_get_tuning(ctx.h, ctypes.byref(t), ctypes.byref(m), ctypes.byref(c)))
    return t.value, m.value, c.value


def lbm_last_error(ctx):
    return load().lbm_last_error(ctx.h).decode()


def lbm_mass_momentum_noalloc(model, storage, f_ptr, nblocks, out_ptr, stream=None):
    """Float64 mass/momentum sums of a caller-owned device array (library
    storage layout) into a caller-owned device array of 4 doubles, without
    any device allocation (see include/lbm.h).  Pointers are integers (e.g.
    torch.Tensor.data_ptr()); the call is asynchronous on `stream`."""
    if not 1 <= int(nblocks) <= NOALLOC_MAX_BLOCKS:
        raise LbmError(LBM_ERR_ARG, "nblocks=%d outside 1..%d: the static scratch holds one "
                       "partial sum per block" % (int(nblocks), NOALLOC_MAX_BLOCKS))
    st = load().lbm_mass_momentum_noalloc(MODELS[model], STORAGES[storage], c_void_p(int(f_ptr)),
                                          int(nblocks), c_void_p(int(out_ptr)),
                                          None if stream is None else c_void_p(int(stream)))
    if st != LBM_OK:
        raise LbmError(st, "lbm_mass_momentum_noalloc failed")


# ------------------------------------------------------------------ block sharding
class Shard(Context):
    """An lbm_shard handle (the whole grid's sizes, as a Context) and its parts."""


def _scheck(sh, st):
    if st != LBM_OK:
        msg = load().lbm_shard_last_error(sh.h if sh is not None else None)
        raise LbmError(st, msg.decode() if msg else "")


def lbm_shard_plan(nb, nparts, periodic_x=True, refine=(), walls=0, slip=0, outlet=0, nozzle=None):
    """Level-0 block-column cuts of nparts parts: [0, c1, ..., nbx]."""
    g, keep = make_grid(nb, periodic_x, refine, walls, slip, outlet, nozzle)
    cuts = (c_int * (nparts + 1))()
    st = load().lbm_shard_plan(ctypes.byref(g), int(nparts), cuts)
    if st != LBM_OK:
        raise LbmError(st, "no admissible cuts")
    return list(cuts)


def lbm_shard_create(model, storage, nb, periodic_x=True, refine=(), omega=1.0, cs=0.0, nparts=2, stream=None,
                     walls=0, slip=0, outlet=0, nozzle=None):
    lib = load()
    g, keep = make_grid(nb, periodic_x, refine, walls, slip, outlet, nozzle)
    h = c_void_p()
    st = lib.lbm_shard_create(ctypes.byref(h), MODELS[model], STORAGES[storage], ctypes.byref(g), float(omega),
                              float(cs), int(nparts), stream)
    if st != LBM_OK:
        raise LbmError(st, lib.lbm_create_error().decode())
    sh = Shard(h, model, nb, g.levels)
    sh.nparts = int(nparts)
    return sh


def lbm_shard_destroy(sh):
    if sh is not None and sh.h:
        load().lbm_shard_destroy(sh.h)
        sh.h = None


def lbm_shard_part(sh, part):
    """(Context of the part, first level-0 column, one past its last)."""
    h, c0, c1 = c_void_p(), c_int(), c_int()
    _scheck(sh, load().lbm_shard_part(sh.h, int(part), ctypes.byref(h), ctypes.byref(c0), ctypes.byref(c1)))
    nb = (c1.value - c0.value, sh.nb[1], sh.nb[2])
    return Context(h, sh.model, nb, sh.levels), c0.value, c1.value


def lbm_shard_halo_bytes(sh):
    n = c_int64()
    _scheck(sh, load().lbm_shard_halo_bytes(sh.h, ctypes.byref(n)))
    return int(n.value)


def lbm_shard_set_inflow(sh, y0, z0, diameter, u_in, perturb=0.01, seed=0):
    _scheck(sh, load().lbm_shard_set_inflow(sh.h, y0, z0, diameter, u_in, perturb, int(seed)))


def lbm_shard_init_equilibrium(sh, level, rho=None, u=None):
    r, v = _f64(rho), _f64(u)
    _scheck(sh, load().lbm_shard_init_equilibrium(sh.h, level, _dptr(r), _dptr(v)))


def lbm_shard_step(sh, n=1):
    _scheck(sh, load().lbm_shard_step(sh.h, int(n)))


def lbm_shard_sync(sh):
    _scheck(sh, load().lbm_shard_sync(sh.h))


def lbm_shard_get_state(sh, level):
    NX, NY, NZ = sh.dims(level)
    f = np.empty((sh.Q, NZ, NY, NX))
    _scheck(sh, load().lbm_shard_get_state(sh.h, level, _dptr(f), f.size))
    return f


def lbm_shard_macroscopic(sh, level):
    NX, NY, NZ = sh.dims(level)
    rho = np.empty((NZ, NY, NX))
    u = np.empty((3, NZ, NY, NX))
    _scheck(sh, load().lbm_shard_macroscopic(sh.h, level, _dptr(rho), _dptr(u)))
    return rho, u


def lbm_shard_mass_momentum(sh):
    out = np.empty(4)
    _scheck(sh, load().lbm_shard_mass_momentum(sh.h, _dptr(out)))
    return out
