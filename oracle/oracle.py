"""ctypes front end of the FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is the plain reference the CUDA library
is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It imports nothing
from the CUDA package.

The oracle follows Algorithm 1 (MEM) and Algorithm 2 (PSM) of Rettinger &
Ruede (arXiv:1702.04910), Sec. 2, literally and in FP64; see the header of
``lbm_oracle.c`` for the readings of points the paper leaves open.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

# coupling and collision codes of the oracle (same meaning as the paper's names)
PSM_M1B1, PSM_M2B2, PSM_M3B2, MEM_BB, MEM_CLI, MEM_MR, NONE = range(7)
BGK, TRT = 0, 1
COUPLING_CODES = {"PSM_M1B1": PSM_M1B1, "PSM_M2B2": PSM_M2B2, "PSM_M3B2": PSM_M3B2,
                  "MEM_BB": MEM_BB, "MEM_CLI": MEM_CLI, "MEM_MR": MEM_MR, "NONE": NONE}
NQ = 19


class Params(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
                ("bc_z", ct.c_int), ("collision", ct.c_int), ("coupling", ct.c_int),
                ("tau", ct.c_double), ("magic", ct.c_double),
                ("fext", ct.c_double * 3), ("gravity", ct.c_double * 3),
                ("rho0", ct.c_double), ("subsample", ct.c_int),
                ("subcycles", ct.c_int), ("wall_contact", ct.c_int),
                ("inflow", ct.c_double * 3), ("rho_out", ct.c_double),
                ("remap_charge", ct.c_int)]


class Particle(ct.Structure):
    _fields_ = [("x", ct.c_double * 3), ("u", ct.c_double * 3),
                ("omega", ct.c_double * 3), ("diameter", ct.c_double),
                ("density", ct.c_double), ("fixed", ct.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ct.CDLL(build())
        P = ct.c_void_p
        dp = ct.POINTER(ct.c_double)
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [ct.POINTER(Params)]
        lib.orc_destroy.argtypes = [P]
        lib.orc_set_particles.argtypes = [P, ct.c_int, ct.POINTER(Particle)]
        lib.orc_get_particles.argtypes = [P, ct.POINTER(Particle)]
        lib.orc_move_and_refill.argtypes = [P, ct.c_int, ct.POINTER(Particle)]
        lib.orc_get_charge.argtypes = [P, dp]
        lib.orc_init_equilibrium.argtypes = [P, ct.c_double, dp]
        lib.orc_set_pdf.argtypes = [P, dp]
        lib.orc_step.argtypes = [P, ct.c_int]
        lib.orc_get_forces.argtypes = [P, dp, dp]
        lib.orc_get_pdf.argtypes = [P, ct.c_int, dp]
        lib.orc_get_macro.argtypes = [P, dp, dp]
        lib.orc_get_solid.argtypes = [P, ct.POINTER(ct.c_int)]
        lib.orc_get_eps.argtypes = [P, ct.c_int, dp]
        lib.orc_feq.restype = ct.c_double
        lib.orc_feq.argtypes = [ct.c_int, ct.c_double, dp, ct.c_double]
        lib.orc_lattice.argtypes = [ct.POINTER(ct.c_int), dp, ct.POINTER(ct.c_int)]
        lib.orc_lambda_minus.restype = ct.c_double
        lib.orc_lambda_minus.argtypes = [P]
        lib.orc_mr_link.restype = ct.c_double
        lib.orc_mr_link.argtypes = [ct.c_double] * 9
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def lattice():
    """(c[19,3], w[19], opp[19]) of the oracle's D3Q19 table."""
    lib = _load()
    c = np.zeros((NQ, 3), dtype=np.int32)
    w = np.zeros(NQ)
    opp = np.zeros(NQ, dtype=np.int32)
    lib.orc_lattice(c.ctypes.data_as(ct.POINTER(ct.c_int)), _dp(w),
                    opp.ctypes.data_as(ct.POINTER(ct.c_int)))
    return c, w, opp


def feq(q: int, rho: float, U, rho0: float = 1.0) -> float:
    """Eq. (3) of the paper, evaluated by the oracle."""
    u = np.ascontiguousarray(U, dtype=np.float64)
    return _load().orc_feq(int(q), float(rho), _dp(u), float(rho0))


def mr_link(delta, Lambda_m, ft_q0, ft_q1, ft_q2, ft_qb0, ft_qb1, n_minus, e_wall) -> float:
    """Eq. (15) multi-reflection value f_qbar(x, t+1) of one link, with the
    coefficients the oracle derives for it (reading R17 of the C file)."""
    return _load().orc_mr_link(*(float(v) for v in (delta, Lambda_m, ft_q0, ft_q1, ft_q2,
                                                       ft_qb0, ft_qb1, n_minus, e_wall)))


class Oracle:
    """One simulation held by the C oracle.

    ``shape`` is (nx, ny, nz); PDF arrays are (19, nz, ny, nx) float64 (SoA,
    x fastest), the layout the CUDA library uses for its field exchange.
    """

    def __init__(self, shape, *, coupling="NONE", collision="TRT", tau=0.8,
                 magic=3.0 / 16.0, fext=(0.0, 0.0, 0.0), gravity=(0.0, 0.0, 0.0),
                 rho0=1.0, bc_z=0, subsample=4, subcycles=0, wall_contact=0,
                 inflow=(0.0, 0.0, 0.0), rho_out=1.0, remap_charge=0):
        self._lib = _load()
        nx, ny, nz = (int(v) for v in shape)
        self.shape = (nx, ny, nz)
        self.coupling = COUPLING_CODES[coupling] if isinstance(coupling, str) else int(coupling)
        p = Params()
        p.nx, p.ny, p.nz = nx, ny, nz
        p.bc_z = int(bc_z)
        p.collision = (TRT if collision == "TRT" else BGK) if isinstance(collision, str) else int(collision)
        p.coupling = self.coupling
        p.tau, p.magic = float(tau), float(magic)
        for a in range(3):
            p.fext[a] = float(fext[a])
            p.gravity[a] = float(gravity[a])
        p.rho0 = float(rho0)
        p.subsample, p.subcycles, p.wall_contact = int(subsample), int(subcycles), int(wall_contact)
        for a in range(3):
            p.inflow[a] = float(inflow[a])
        p.rho_out = float(rho_out)
        p.remap_charge = int(remap_charge)
        self.params = p
        h = self._lib.orc_create(ct.byref(p))
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = ct.c_void_p(h)
        self.np = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

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
    def lambda_minus(self):
        return self._lib.orc_lambda_minus(self._h)

    @staticmethod
    def _records(particles):
        arr = (Particle * max(1, len(particles)))()
        for i, d in enumerate(particles):
            for a in range(3):
                arr[i].x[a] = float(d["x"][a])
                arr[i].u[a] = float(d.get("u", (0, 0, 0))[a])
                arr[i].omega[a] = float(d.get("omega", (0, 0, 0))[a])
            arr[i].diameter = float(d["diameter"])
            arr[i].density = float(d.get("density", 1.0))
            arr[i].fixed = int(d.get("fixed", 0))
        return arr

    def set_particles(self, particles):
        """particles: list of dicts with x, u, omega, diameter, density, fixed."""
        arr = self._records(particles)
        st = self._lib.orc_set_particles(self._h, len(particles), arr)
        if st != 0:
            raise ValueError(f"oracle set_particles failed ({st})")
        self.np = len(particles)

    def move_and_refill(self, particles):
        """MEM only: give the mapped particles a new state (as a rigid-body
        update would) and run the re-mapping and PDF reconstruction of
        Sec. 2.2 alone on the current pre-collision field.  The momentum
        amounts of the re-mapping (R32) are kept as the pending charge
        (``charge()``) whether or not the option is on."""
        st = self._lib.orc_move_and_refill(self._h, len(particles), self._records(particles))
        if st != 0:
            raise ValueError(f"oracle move_and_refill failed ({st})")

    def get_particles(self):
        arr = (Particle * max(1, self.np))()
        self._lib.orc_get_particles(self._h, arr)
        out = []
        for i in range(self.np):
            out.append({"x": np.array(arr[i].x[:]), "u": np.array(arr[i].u[:]),
                        "omega": np.array(arr[i].omega[:]), "diameter": arr[i].diameter,
                        "density": arr[i].density, "fixed": arr[i].fixed})
        return out

    def init_equilibrium(self, rho=1.0, u=(0.0, 0.0, 0.0)):
        uu = np.ascontiguousarray(u, dtype=np.float64)
        self._lib.orc_init_equilibrium(self._h, float(rho), _dp(uu))

    def set_pdf(self, f_pre: np.ndarray):
        """Set the pre-collision PDF field f (19, nz, ny, nx)."""
        f = np.ascontiguousarray(f_pre, dtype=np.float64)
        assert f.size == NQ * self.ncells
        self._lib.orc_set_pdf(self._h, _dp(f))

    def step(self, n=1):
        st = self._lib.orc_step(self._h, int(n))
        return st

    def charge(self):
        """R32: (np, 6) momentum and angular momentum (about the new centre)
        that the last re-mapping gave the fluid: uncovered minus covered
        cells.  With remap_charge = 1 the next step takes charge / dt off the
        force and torque."""
        out = np.zeros((max(1, self.np), 6))
        self._lib.orc_get_charge(self._h, _dp(out))
        return out[: self.np]

    def forces(self):
        F = np.zeros((max(1, self.np), 3))
        T = np.zeros((max(1, self.np), 3))
        self._lib.orc_get_forces(self._h, _dp(F), _dp(T))
        return F[: self.np], T[: self.np]

    def pdf(self, which="post"):
        """'pre' current pre-collision f; 'post' last post-collision f~;
        'collide' the post-collision values of a plain fluid collision of the
        current f (Eq. 1)."""
        code = {"pre": 0, "post": 1, "collide": 2}[which]
        nx, ny, nz = self.shape
        out = np.zeros((NQ, nz, ny, nx))
        self._lib.orc_get_pdf(self._h, code, _dp(out))
        return out

    def macro(self):
        nx, ny, nz = self.shape
        rho = np.zeros((nz, ny, nx))
        u = np.zeros((nz, ny, nx, 3))
        self._lib.orc_get_macro(self._h, _dp(rho), _dp(u))
        return rho, u

    def solid(self):
        nx, ny, nz = self.shape
        out = np.zeros((nz, ny, nx), dtype=np.int32)
        self._lib.orc_get_solid(self._h, out.ctypes.data_as(ct.POINTER(ct.c_int)))
        return out

    def eps(self, p=0):
        nx, ny, nz = self.shape
        out = np.zeros((nz, ny, nx))
        self._lib.orc_get_eps(self._h, int(p), _dp(out))
        return out
