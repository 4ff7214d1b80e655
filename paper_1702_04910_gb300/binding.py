"""Thin ctypes binding of ``liblbm_gb300.so`` (C ABI in ``include/lbm_gb300.h``).

Argument marshalling only: every step of the coupled lattice Boltzmann path
runs in the CUDA library.  There is no fallback: if the library is missing or
cannot be loaded, :func:`load` raises.

The module-level functions carry the C names (``lbm_create``, ``lbm_step``,
...).  :class:`Simulation` bundles a handle with NumPy / torch-friendly
marshalling for the tests and the benchmark.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np

from . import build as _build

NQ = 19

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM = 0, -1, -2, -3
LBM_ERR_UNSTABLE, LBM_ERR_DOMAIN, LBM_ERR_TIMEOUT, LBM_ERR_UNSUPPORTED = -4, -5, -6, -7
STATUS_NAMES = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_OOM",
                -4: "LBM_ERR_UNSTABLE", -5: "LBM_ERR_DOMAIN", -6: "LBM_ERR_TIMEOUT",
                -7: "LBM_ERR_UNSUPPORTED"}
# bits kernels OR into a device status word (lbm_sweep_noalloc's status_dev)
STATUS_BITS = {"LBM_STATUS_TOO_MANY_OBJECTS": 1, "LBM_STATUS_DOMAIN": 2, "LBM_STATUS_UNSTABLE": 8,
               "LBM_STATUS_BOUNDS": 16, "LBM_STATUS_FLUID": 32}

COUPLING = {"PSM_M1B1": 0, "PSM_M2B2": 1, "PSM_M3B2": 2, "MEM_BB": 3, "MEM_CLI": 4,
            "MEM_MR": 5, "NONE": 6}
COLLISION = {"BGK": 0, "TRT": 1}
STORAGE = {"f64": 0, "f32": 1, "f64ff": 2, "f64fx": 3, "f16s": 4, "bf16s": 5}
(FIELD_PDF, FIELD_PDF_PRE, FIELD_RHO, FIELD_U, FIELD_EPS, FIELD_FLAG, FIELD_PDF_F64,
 FIELD_REMAP_CHARGE) = range(8)
PROFILE_CLASSES = ("bulk", "near", "force_total", "rigid_body", "refill", "other")

EXPORTED = ("lbm_create", "lbm_set_particles", "lbm_get_particles", "lbm_init_equilibrium",
            "lbm_step", "lbm_get_forces", "lbm_get_fields", "lbm_set_fields",
            "lbm_synchronize", "lbm_profile_enable", "lbm_profile_read", "lbm_device_bytes",
            "lbm_destroy", "lbm_last_error", "lbm_abi_version", "lbm_sweep_noalloc",
            "lbm_batch_create", "lbm_batch_step", "lbm_batch_autotune", "lbm_batch_set_tuning",
            "lbm_batch_get_particles", "lbm_batch_get_forces", "lbm_batch_get_pdf",
            "lbm_batch_cell_updates", "lbm_batch_device_bytes", "lbm_batch_graph_kernels",
            "lbm_batch_synchronize", "lbm_batch_destroy", "lbm_batch_last_error",
            "lbm_mlp_create", "lbm_mlp_destroy", "lbm_mlp_last_error", "lbm_mlp_set_params",
            "lbm_mlp_get_params", "lbm_mlp_set_normalization", "lbm_mlp_get_normalization",
            "lbm_mlp_fit_normalization", "lbm_mlp_forward", "lbm_mlp_gradient", "lbm_mlp_train",
            "lbm_set_force_model", "lbm_get_features", "lbm_measure_fp64_rate",
            "lbm_set_remap_charge", "lbm_batch_profile_enable", "lbm_batch_profile_read",
            "lbm_batch_set_remap_charge")
MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_PARAMS, MLP_NORM = 512, 64, 6, 37382, 1030
BATCH_LAYOUTS = {"box32": 0, "box64": 1, "box128": 2, "plane": 3}


class LbmConfig(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int), ("bc_z", ct.c_int),
                ("collision", ct.c_int), ("coupling", ct.c_int), ("tau", ct.c_double),
                ("magic", ct.c_double), ("force_density", ct.c_double * 3),
                ("gravity", ct.c_double * 3), ("rho0", ct.c_double), ("subsample", ct.c_int),
                ("lbm_subcycles", ct.c_int), ("wall_contact", ct.c_int), ("storage", ct.c_int),
                ("inflow", ct.c_double * 3), ("rho_out", ct.c_double)]


class LbmParticle(ct.Structure):
    _fields_ = [("x", ct.c_double * 3), ("u", ct.c_double * 3), ("omega", ct.c_double * 3),
                ("diameter", ct.c_double), ("density", ct.c_double), ("fixed", ct.c_int)]


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if allowed and missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library {path} is not built")
            _build.build()
        lib = ct.CDLL(path)
        vp, dp, i, sz = ct.c_void_p, ct.POINTER(ct.c_double), ct.c_int, ct.c_size_t
        fp = ct.POINTER(ct.c_float)
        sig = {
            "lbm_create": (i, [ct.POINTER(LbmConfig), vp, ct.POINTER(vp)]),
            "lbm_set_particles": (i, [vp, i, ct.POINTER(LbmParticle)]),
            "lbm_get_particles": (i, [vp, ct.POINTER(LbmParticle)]),
            "lbm_init_equilibrium": (i, [vp, ct.c_double, dp]),
            "lbm_step": (i, [vp, i]),
            "lbm_get_forces": (i, [vp, dp, dp]),
            "lbm_get_fields": (i, [vp, i, vp, sz, i]),
            "lbm_set_fields": (i, [vp, i, vp, sz, i]),
            "lbm_synchronize": (i, [vp]),
            "lbm_profile_enable": (i, [vp, i]),
            "lbm_profile_read": (i, [vp, i, dp, ct.POINTER(ct.c_longlong)]),
            "lbm_device_bytes": (sz, [vp]),
            "lbm_destroy": (None, [vp]),
            "lbm_last_error": (ct.c_char_p, [vp]),
            "lbm_abi_version": (i, []),
            "lbm_sweep_noalloc": (i, [ct.POINTER(LbmConfig), vp, vp, i, ct.POINTER(LbmParticle),
                                      vp, vp, vp, ct.c_char_p, sz]),
            "lbm_batch_create": (i, [i, ct.POINTER(LbmConfig), ct.POINTER(LbmParticle), vp,
                                     ct.POINTER(vp)]),
            "lbm_batch_step": (i, [vp, i]),
            "lbm_batch_autotune": (i, [vp, i, ct.POINTER(i), ct.POINTER(i), dp]),
            "lbm_batch_set_tuning": (i, [vp, ct.POINTER(i), i]),
            "lbm_batch_get_particles": (i, [vp, ct.POINTER(LbmParticle)]),
            "lbm_batch_get_forces": (i, [vp, dp, dp]),
            "lbm_batch_get_pdf": (i, [vp, i, dp, sz]),
            "lbm_batch_cell_updates": (ct.c_longlong, [vp]),
            "lbm_batch_device_bytes": (sz, [vp]),
            "lbm_batch_graph_kernels": (i, [vp]),
            "lbm_batch_profile_enable": (i, [vp, i]),
            "lbm_batch_set_remap_charge": (i, [vp, i]),
            "lbm_batch_profile_read": (i, [vp, ct.POINTER(ct.c_double), ct.POINTER(ct.c_longlong)]),
            "lbm_batch_synchronize": (i, [vp]),
            "lbm_batch_destroy": (None, [vp]),
            "lbm_batch_last_error": (ct.c_char_p, [vp]),
            "lbm_mlp_create": (i, [vp, ct.POINTER(vp)]),
            "lbm_mlp_destroy": (None, [vp]),
            "lbm_mlp_last_error": (ct.c_char_p, [vp]),
            "lbm_mlp_set_params": (i, [vp, fp, sz]),
            "lbm_mlp_get_params": (i, [vp, fp, sz]),
            "lbm_mlp_set_normalization": (i, [vp, fp, sz]),
            "lbm_mlp_get_normalization": (i, [vp, fp, sz]),
            "lbm_mlp_fit_normalization": (i, [vp, vp, vp, i]),
            "lbm_mlp_forward": (i, [vp, vp, i, vp]),
            "lbm_mlp_gradient": (i, [vp, vp, vp, i, fp, sz, dp]),
            "lbm_mlp_train": (i, [vp, vp, vp, i, i, ct.c_float, dp]),
            "lbm_set_force_model": (i, [vp, vp, ct.c_double, i]),
            "lbm_set_remap_charge": (i, [vp, i]),
            "lbm_get_features": (i, [vp, fp, sz]),
            "lbm_measure_fp64_rate": (i, [vp, dp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


# ---- C-named entry points (marshalling only) -------------------------------------
def _check(h, st):
    if st != LBM_OK:
        msg = load().lbm_last_error(h)
        raise LbmError(st, msg.decode() if msg else "")
    return st


def make_config(shape, *, coupling="NONE", collision="TRT", tau=0.8, magic=3.0 / 16.0,
                fext=(0.0, 0.0, 0.0), gravity=(0.0, 0.0, 0.0), rho0=1.0, bc_z=0, subsample=4,
                subcycles=0, wall_contact=0, storage="f64", inflow=(0.0, 0.0, 0.0),
                rho_out=1.0) -> LbmConfig:
    c = LbmConfig()
    c.nx, c.ny, c.nz = (int(v) for v in shape)
    c.bc_z = int(bc_z)
    c.collision = COLLISION[collision] if isinstance(collision, str) else int(collision)
    c.coupling = COUPLING[coupling] if isinstance(coupling, str) else int(coupling)
    c.tau, c.magic = float(tau), float(magic)
    for a in range(3):
        c.force_density[a] = float(fext[a])
        c.gravity[a] = float(gravity[a])
    c.rho0 = float(rho0)
    c.subsample, c.lbm_subcycles, c.wall_contact = int(subsample), int(subcycles), int(wall_contact)
    c.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    for a in range(3):
        c.inflow[a] = float(inflow[a])
    c.rho_out = float(rho_out)
    return c


def particles_to_c(particles):
    arr = (LbmParticle * max(1, len(particles)))()
    for i, d in enumerate(particles):
        for a in range(3):
            arr[i].x[a] = float(d["x"][a])
            arr[i].u[a] = float(d.get("u", (0, 0, 0))[a])
            arr[i].omega[a] = float(d.get("omega", (0, 0, 0))[a])
        arr[i].diameter = float(d["diameter"])
        arr[i].density = float(d.get("density", 1.0))
        arr[i].fixed = int(d.get("fixed", 0))
    return arr


def lbm_create(cfg: LbmConfig, stream: int | None = None) -> ct.c_void_p:
    lib = load()
    h = ct.c_void_p()
    st = lib.lbm_create(ct.byref(cfg), ct.c_void_p(stream or 0), ct.byref(h))
    if st != LBM_OK:
        raise LbmError(st, "lbm_create rejected the configuration")
    return h


def lbm_destroy(h) -> None:
    load().lbm_destroy(h)


def lbm_set_particles(h, particles) -> None:
    _check(h, load().lbm_set_particles(h, len(particles), particles_to_c(particles)))


def lbm_get_particles(h, n: int):
    arr = (LbmParticle * max(1, n))()
    _check(h, load().lbm_get_particles(h, arr))
    return [{"x": np.array(arr[i].x[:]), "u": np.array(arr[i].u[:]),
             "omega": np.array(arr[i].omega[:]), "diameter": arr[i].diameter,
             "density": arr[i].density, "fixed": arr[i].fixed} for i in range(n)]


def lbm_init_equilibrium(h, rho: float, u) -> None:
    uu = np.ascontiguousarray(u, dtype=np.float64)
    _check(h, load().lbm_init_equilibrium(h, float(rho), uu.ctypes.data_as(ct.POINTER(ct.c_double))))


def lbm_step(h, nsteps: int) -> None:
    _check(h, load().lbm_step(h, int(nsteps)))


def lbm_get_forces(h, n: int, F: np.ndarray | None = None, T: np.ndarray | None = None):
    F = np.zeros((max(n, 1), 3)) if F is None else F
    T = np.zeros((max(n, 1), 3)) if T is None else T
    _check(h, load().lbm_get_forces(h, F.ctypes.data_as(ct.POINTER(ct.c_double)),
                                    T.ctypes.data_as(ct.POINTER(ct.c_double))))
    return F[:n], T[:n]


def lbm_get_fields(h, what: int, ptr: int, nbytes: int, is_device: bool) -> None:
    _check(h, load().lbm_get_fields(h, int(what), ct.c_void_p(ptr), nbytes, int(is_device)))


def lbm_set_fields(h, what: int, ptr: int, nbytes: int, is_device: bool) -> None:
    _check(h, load().lbm_set_fields(h, int(what), ct.c_void_p(ptr), nbytes, int(is_device)))


def lbm_synchronize(h) -> None:
    _check(h, load().lbm_synchronize(h))


def lbm_profile_enable(h, enable: bool) -> None:
    _check(h, load().lbm_profile_enable(h, int(bool(enable))))


def lbm_profile_read(h):
    n = len(PROFILE_CLASSES)
    ms = (ct.c_double * n)()
    cnt = (ct.c_longlong * n)()
    _check(h, load().lbm_profile_read(h, n, ms, cnt))
    return {PROFILE_CLASSES[k]: (ms[k], cnt[k]) for k in range(n)}


def lbm_sweep_noalloc(cfg: LbmConfig, src_ptr: int, dst_ptr: int, particles, ft_ptr: int,
                      status_ptr: int = 0, stream: int | None = None) -> None:
    """One coupled sweep on caller-owned device buffers (no allocation)."""
    arr = particles_to_c(particles)
    err = ct.create_string_buffer(256)
    st = load().lbm_sweep_noalloc(ct.byref(cfg), ct.c_void_p(src_ptr), ct.c_void_p(dst_ptr),
                                  len(particles), arr, ct.c_void_p(ft_ptr or None),
                                  ct.c_void_p(status_ptr or None), ct.c_void_p(stream or 0),
                                  err, len(err))
    if st != LBM_OK:
        raise LbmError(st, err.value.decode())


def lbm_device_bytes(h) -> int:
    return int(load().lbm_device_bytes(h))


# ---- batched ensemble (C names) ------------------------------------------------------
def _bcheck(b, st):
    if st != LBM_OK:
        msg = load().lbm_batch_last_error(b)
        raise LbmError(st, msg.decode() if msg else "")
    return st


def lbm_batch_create(cfgs, particles, stream: int | None = None) -> ct.c_void_p:
    """cfgs: list of LbmConfig; particles: one particle dict per case."""
    n = len(cfgs)
    carr = (LbmConfig * n)(*cfgs)
    parr = particles_to_c(particles)
    b = ct.c_void_p()
    _bcheck(None, load().lbm_batch_create(n, carr, parr, ct.c_void_p(stream or 0), ct.byref(b)))
    return b


def lbm_batch_step(b, nsteps: int) -> None:
    _bcheck(b, load().lbm_batch_step(b, int(nsteps)))


def lbm_batch_autotune(b, n: int, reps: int = 5):
    """Returns (per-case layouts, grid, bulk ms)."""
    lays = (ct.c_int * n)()
    grid, ms = ct.c_int(), ct.c_double()
    _bcheck(b, load().lbm_batch_autotune(b, int(reps), lays, ct.byref(grid), ct.byref(ms)))
    return list(lays), grid.value, ms.value


def lbm_batch_set_tuning(b, layouts, grid: int) -> None:
    """layouts: one LBM_BATCH_* code per case, or None (all plane)."""
    arr = None if layouts is None else (ct.c_int * len(layouts))(*[int(v) for v in layouts])
    _bcheck(b, load().lbm_batch_set_tuning(b, arr, int(grid)))


def lbm_batch_get_particles(b, n: int):
    arr = (LbmParticle * n)()
    _bcheck(b, load().lbm_batch_get_particles(b, arr))
    return [{"x": np.array(arr[i].x[:]), "u": np.array(arr[i].u[:]),
             "omega": np.array(arr[i].omega[:]), "diameter": arr[i].diameter,
             "density": arr[i].density, "fixed": arr[i].fixed} for i in range(n)]


def lbm_batch_get_forces(b, n: int):
    F = np.zeros((n, 3))
    T = np.zeros((n, 3))
    _bcheck(b, load().lbm_batch_get_forces(b, F.ctypes.data_as(ct.POINTER(ct.c_double)),
                                           T.ctypes.data_as(ct.POINTER(ct.c_double))))
    return F, T


def lbm_batch_get_pdf(b, c: int, shape) -> np.ndarray:
    nx, ny, nz = shape
    out = np.empty((NQ, nz, ny, nx))
    _bcheck(b, load().lbm_batch_get_pdf(b, int(c), out.ctypes.data_as(ct.POINTER(ct.c_double)),
                                        out.nbytes))
    return out


def lbm_batch_cell_updates(b) -> int:
    return int(load().lbm_batch_cell_updates(b))


def lbm_batch_device_bytes(b) -> int:
    return int(load().lbm_batch_device_bytes(b))


def lbm_batch_graph_kernels(b) -> int:
    return int(load().lbm_batch_graph_kernels(b))


def lbm_batch_synchronize(b) -> None:
    _bcheck(b, load().lbm_batch_synchronize(b))


def lbm_batch_set_remap_charge(b, enable: int) -> None:
    _bcheck(b, load().lbm_batch_set_remap_charge(b, int(enable)))


def lbm_batch_profile_enable(b, enable: int) -> None:
    _bcheck(b, load().lbm_batch_profile_enable(b, int(enable)))


def lbm_batch_profile_read(b):
    ms, n = ct.c_double(), ct.c_longlong()
    _bcheck(b, load().lbm_batch_profile_read(b, ct.byref(ms), ct.byref(n)))
    return ms.value, n.value


def lbm_batch_destroy(b) -> None:
    load().lbm_batch_destroy(b)


# ---- learned force correction (C names) ---------------------------------------------
def _mcheck(m, st):
    if st != LBM_OK:
        msg = load().lbm_mlp_last_error(m)
        raise LbmError(st, msg.decode() if msg else "")
    return st


def _fptr(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(ct.POINTER(ct.c_float))


def lbm_mlp_create(stream: int | None = None) -> ct.c_void_p:
    m = ct.c_void_p()
    st = load().lbm_mlp_create(ct.c_void_p(stream or 0), ct.byref(m))
    if st != LBM_OK:
        raise LbmError(st, "lbm_mlp_create failed")
    return m


def lbm_mlp_destroy(m) -> None:
    load().lbm_mlp_destroy(m)


def lbm_mlp_set_params(m, params: np.ndarray) -> None:
    a = np.ascontiguousarray(params, dtype=np.float32)
    _mcheck(m, load().lbm_mlp_set_params(m, _fptr(a), a.size))


def lbm_mlp_get_params(m) -> np.ndarray:
    a = np.empty(MLP_PARAMS, dtype=np.float32)
    _mcheck(m, load().lbm_mlp_get_params(m, _fptr(a), a.size))
    return a


def lbm_mlp_set_normalization(m, norm: np.ndarray) -> None:
    a = np.ascontiguousarray(norm, dtype=np.float32)
    _mcheck(m, load().lbm_mlp_set_normalization(m, _fptr(a), a.size))


def lbm_mlp_get_normalization(m) -> np.ndarray:
    a = np.empty(MLP_NORM, dtype=np.float32)
    _mcheck(m, load().lbm_mlp_get_normalization(m, _fptr(a), a.size))
    return a


def lbm_mlp_fit_normalization(m, x_ptr: int, t_ptr: int, n: int) -> None:
    _mcheck(m, load().lbm_mlp_fit_normalization(m, ct.c_void_p(x_ptr), ct.c_void_p(t_ptr), int(n)))


def lbm_mlp_forward(m, x_ptr: int, n: int, y_ptr: int) -> None:
    _mcheck(m, load().lbm_mlp_forward(m, ct.c_void_p(x_ptr), int(n), ct.c_void_p(y_ptr)))


def lbm_mlp_gradient(m, x_ptr: int, t_ptr: int, n: int):
    g = np.empty(MLP_PARAMS, dtype=np.float32)
    loss = ct.c_double()
    _mcheck(m, load().lbm_mlp_gradient(m, ct.c_void_p(x_ptr), ct.c_void_p(t_ptr), int(n), _fptr(g),
                                       g.size, ct.byref(loss)))
    return g, loss.value


def lbm_mlp_train(m, x_ptr: int, t_ptr: int, n: int, steps: int, lr: float) -> float:
    loss = ct.c_double()
    _mcheck(m, load().lbm_mlp_train(m, ct.c_void_p(x_ptr), ct.c_void_p(t_ptr), int(n), int(steps),
                                    float(lr), ct.byref(loss)))
    return loss.value


def lbm_set_force_model(h, m, u_ref: float, mode: int) -> None:
    _check(h, load().lbm_set_force_model(h, m, float(u_ref), int(mode)))


def lbm_set_remap_charge(h, enable: int) -> None:
    _check(h, load().lbm_set_remap_charge(h, int(enable)))


def lbm_get_features(h, n: int) -> np.ndarray:
    a = np.empty((n, MLP_IN), dtype=np.float32)
    _check(h, load().lbm_get_features(h, _fptr(a), a.size))
    return a


def lbm_measure_fp64_rate(stream: int | None = None) -> float:
    """Measured FP64 fused multiply-add lane-operations per second of the
    current device (the FP64 roofline of the sweep)."""
    out = ct.c_double(0.0)
    st = load().lbm_measure_fp64_rate(ct.c_void_p(stream or 0), ct.byref(out))
    if st != LBM_OK:
        raise LbmError(st, "FP64 rate probe failed")
    return out.value


# ---- convenience wrapper ------------------------------------------------------------
class Simulation:
    """One library handle; arrays are NumPy (host) unless noted."""

    def __init__(self, shape, stream: int | None = None, **kw):
        self.shape = tuple(int(v) for v in shape)
        self.storage = kw.get("storage", "f64")
        self.cfg = make_config(shape, **kw)
        self.h = lbm_create(self.cfg, stream)
        self.np = 0

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ncells(self):
        nx, ny, nz = self.shape
        return nx * ny * nz

    @property
    def pdf_dtype(self):
        """NumPy dtype of the stored PDF array (16-bit formats: raw bits)."""
        return {"f32": np.float32, "f16s": np.float16, "bf16s": np.uint16}.get(self.storage,
                                                                               np.float64)

    def pdf_f64(self) -> np.ndarray:
        """Stored post-collision PDFs as FP64 values of f (converted on the GPU)."""
        nx, ny, nz = self.shape
        out = np.empty((NQ, nz, ny, nx), dtype=np.float64)
        lbm_get_fields(self.h, FIELD_PDF_F64, out.ctypes.data, out.nbytes, False)
        return out

    def set_particles(self, particles):
        lbm_set_particles(self.h, particles)
        self.np = len(particles)

    def get_particles(self):
        return lbm_get_particles(self.h, self.np)

    def init_equilibrium(self, rho=1.0, u=(0.0, 0.0, 0.0)):
        lbm_init_equilibrium(self.h, rho, u)

    def step(self, n=1):
        lbm_step(self.h, n)

    def forces(self):
        return lbm_get_forces(self.h, self.np)

    def set_pdf_pre(self, f: np.ndarray):
        a = np.ascontiguousarray(f, dtype=np.float64)
        assert a.size == NQ * self.ncells
        lbm_set_fields(self.h, FIELD_PDF_PRE, a.ctypes.data, a.nbytes, False)

    def pdf(self) -> np.ndarray:
        nx, ny, nz = self.shape
        out = np.empty((NQ, nz, ny, nx), dtype=self.pdf_dtype)
        lbm_get_fields(self.h, FIELD_PDF, out.ctypes.data, out.nbytes, False)
        return out

    def set_pdf(self, f: np.ndarray):
        a = np.ascontiguousarray(f, dtype=self.pdf_dtype)
        lbm_set_fields(self.h, FIELD_PDF, a.ctypes.data, a.nbytes, False)

    def macro(self):
        nx, ny, nz = self.shape
        rho = np.empty((nz, ny, nx))
        u = np.empty((nz, ny, nx, 3))
        lbm_get_fields(self.h, FIELD_RHO, rho.ctypes.data, rho.nbytes, False)
        lbm_get_fields(self.h, FIELD_U, u.ctypes.data, u.nbytes, False)
        return rho, u

    def eps(self):
        nx, ny, nz = self.shape
        out = np.empty((nz, ny, nx))
        lbm_get_fields(self.h, FIELD_EPS, out.ctypes.data, out.nbytes, False)
        return out

    def flags(self):
        nx, ny, nz = self.shape
        out = np.empty((nz, ny, nx), dtype=np.int32)
        lbm_get_fields(self.h, FIELD_FLAG, out.ctypes.data, out.nbytes, False)
        return out

    def synchronize(self):
        lbm_synchronize(self.h)

    def set_remap_charge(self, enable=True):
        """MEM: charge the momentum of covered and uncovered cells to the
        particle at the next step (``lbm_set_remap_charge``)."""
        lbm_set_remap_charge(self.h, 1 if enable else 0)

    def remap_charge(self) -> np.ndarray:
        """(np, 6): the pending re-mapping charge (momentum, angular momentum)."""
        out = np.zeros((self.np, 6))
        lbm_get_fields(self.h, FIELD_REMAP_CHARGE, out.ctypes.data, out.nbytes, False)
        return out

    def set_remap_charge_state(self, charge: np.ndarray):
        a = np.ascontiguousarray(charge, dtype=np.float64)
        assert a.size == 6 * self.np
        lbm_set_fields(self.h, FIELD_REMAP_CHARGE, a.ctypes.data, a.nbytes, False)

    def set_force_model(self, model, u_ref, mode=1):
        """model: an :class:`Mlp` (or None with mode 2: features only)."""
        lbm_set_force_model(self.h, model.m if model is not None else None, u_ref, mode)
        self._model = model  # keep it alive while attached

    def features(self):
        return lbm_get_features(self.h, self.np)


class Batch:
    """A batched ensemble: ``cases`` are workload dicts with one particle each
    (shape, solver keywords, particles)."""

    def __init__(self, cases, storage: str = "f64", stream: int | None = None):
        from .workloads import sim_kwargs
        self.shapes = [tuple(int(v) for v in c["shape"]) for c in cases]
        cfgs = [make_config(c["shape"], storage=storage, **sim_kwargs(c)) for c in cases]
        self.n = len(cases)
        self.b = lbm_batch_create(cfgs, [c["particles"][0] for c in cases], stream)

    def close(self):
        if getattr(self, "b", None):
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        lbm_batch_step(self.b, n)

    def autotune(self, reps=5):
        """Per-case layouts (names), grid, bulk ms."""
        lays, grid, ms = lbm_batch_autotune(self.b, self.n, reps)
        names = {v: k for k, v in BATCH_LAYOUTS.items()}
        return [names[v] for v in lays], grid, ms

    def set_tuning(self, layout, grid):
        """layout: a name or code for every case, or a list with one per case."""
        if isinstance(layout, (list, tuple)):
            lays = [BATCH_LAYOUTS.get(v, v) for v in layout]
        else:
            lays = [BATCH_LAYOUTS.get(layout, layout)] * self.n
        lbm_batch_set_tuning(self.b, lays, grid)

    def particles(self):
        return lbm_batch_get_particles(self.b, self.n)

    def forces(self):
        return lbm_batch_get_forces(self.b, self.n)

    def pdf(self, c):
        return lbm_batch_get_pdf(self.b, c, self.shapes[c])

    @property
    def cell_updates(self):
        return lbm_batch_cell_updates(self.b)

    @property
    def device_bytes(self):
        return lbm_batch_device_bytes(self.b)

    @property
    def graph_kernels(self):
        return lbm_batch_graph_kernels(self.b)

    def synchronize(self):
        lbm_batch_synchronize(self.b)

    def set_remap_charge(self, enable=True):
        """MEM cases: charge the re-mapping momentum (``lbm_batch_set_remap_charge``)."""
        lbm_batch_set_remap_charge(self.b, 1 if enable else 0)

    def profile(self, enable=True):
        """Time every bulk sweep on the device from now on (graph rebuilt)."""
        lbm_batch_profile_enable(self.b, 1 if enable else 0)

    def profile_read(self):
        """(summed bulk-sweep milliseconds, bulk sweeps timed)."""
        return lbm_batch_profile_read(self.b)


class Mlp:
    """The force-correction network on the GPU (parameters, normalisation and
    Adam state live on the device; data buffers are passed as device pointers)."""

    def __init__(self, stream: int | None = None):
        self.m = lbm_mlp_create(stream)

    def close(self):
        if getattr(self, "m", None):
            lbm_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        lbm_mlp_set_params(self.m, p)

    def params(self):
        return lbm_mlp_get_params(self.m)

    def set_normalization(self, nrm):
        lbm_mlp_set_normalization(self.m, nrm)

    def normalization(self):
        return lbm_mlp_get_normalization(self.m)

    def fit_normalization(self, x_ptr, t_ptr, n):
        lbm_mlp_fit_normalization(self.m, x_ptr, t_ptr, n)

    def forward(self, x_ptr, n, y_ptr):
        lbm_mlp_forward(self.m, x_ptr, n, y_ptr)

    def gradient(self, x_ptr, t_ptr, n):
        return lbm_mlp_gradient(self.m, x_ptr, t_ptr, n)

    def train(self, x_ptr, t_ptr, n, steps, lr):
        return lbm_mlp_train(self.m, x_ptr, t_ptr, n, steps, lr)
