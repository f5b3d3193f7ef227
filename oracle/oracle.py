"""Python handle on the FP64 CPU oracle (``lbib_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle checks the CUDA path of the coupled
lattice-Boltzmann / immersed-boundary step (arXiv:1606.01805, Section 2).
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` and reference legs import this module.  It imports nothing
from the CUDA package and the package imports nothing from here.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "lbib_oracle.c"
LIB = HERE / "_build" / "liblbib_oracle.so"

PERIODIC, VELOCITY = 0, 1
INIT_REST, INIT_COUETTE, INIT_TAYLOR_GREEN = 0, 1, 2
CIRCLE, ELLIPSE, RECT, SQUARE, TRIANGLE = 0, 1, 2, 3, 4
W_EXP, W_CUBIC, W_QUARTIC, W_COSINE, W_POLY = 0, 1, 2, 3, 4
OK, EINVAL, EDOMAIN = 0, 1, 7


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain C11, no FMA contraction)."""
    LIB.parent.mkdir(parents=True, exist_ok=True)
    if force or not LIB.exists() or LIB.stat().st_mtime < max(
        SRC.stat().st_mtime, (HERE / "lbib_oracle.h").stat().st_mtime
    ):
        tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", str(tmp), str(SRC), "-lm"]
        # OpenMP threads over the rows of the lattice loops, where gcc has it
        if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
            subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


class Config(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("tau", C.c_double),
        ("bc", C.c_int * 4), ("wall_u", (C.c_double * 2) * 4),
        ("body_force", C.c_double * 2), ("gravity", C.c_double * 2),
        ("init", C.c_int), ("init_u", C.c_double), ("weight", C.c_int),
        ("spacing", C.c_double),
    ]


class ParticleDesc(C.Structure):
    _fields_ = [
        ("shape", C.c_int), ("dim", C.c_double * 2), ("xc", C.c_double),
        ("yc", C.c_double), ("theta", C.c_double), ("rho_s", C.c_double),
        ("u0", C.c_double * 2), ("omega0", C.c_double), ("n_markers", C.c_int),
    ]


class ParticleState(C.Structure):
    _fields_ = [
        ("xc", C.c_double), ("yc", C.c_double), ("theta", C.c_double),
        ("u", C.c_double * 2), ("omega", C.c_double), ("F", C.c_double * 2),
        ("M", C.c_double),
    ]


_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(str(build()))
        L.ob_create.restype = C.c_void_p
        L.ob_create.argtypes = [C.POINTER(Config), C.POINTER(C.c_int)]
        L.ob_destroy.argtypes = [C.c_void_p]
        L.ob_add_particle.argtypes = [C.c_void_p, C.POINTER(ParticleDesc)]
        L.ob_step.argtypes = [C.c_void_p, C.c_int]
        L.ob_last_error.restype = C.c_char_p
        L.ob_last_error.argtypes = [C.c_void_p]
        L.ob_steps_done.restype = C.c_long
        L.ob_steps_done.argtypes = [C.c_void_p]
        L.ob_get_populations.argtypes = [C.c_void_p, _dp]
        L.ob_set_populations.argtypes = [C.c_void_p, _dp]
        L.ob_get_fields.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.ob_get_particles.argtypes = [C.c_void_p, C.POINTER(ParticleState), C.c_int]
        L.ob_get_markers.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, C.c_int]
        L.ob_particle_props.argtypes = [C.c_void_p, C.c_int] + [C.POINTER(C.c_double)] * 3
        L.ob_get_force_field.argtypes = [C.c_void_p, _dp]
        L.ob_lattice.argtypes = [_ip, _dp]
        L.ob_feq.argtypes = [C.c_double] * 3 + [_dp]
        L.ob_collide.argtypes = [_dp, C.c_double, C.c_double, C.c_double, _dp]
        L.ob_guo_term.argtypes = [C.c_double] * 5 + [_dp]
        L.ob_mls.argtypes = [C.c_int, C.c_double, C.c_double, _ip, _ip, _dp]
        L.ob_weight.restype = C.c_double
        L.ob_weight.argtypes = [C.c_int, C.c_double]
        L.ob_stress_force.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, C.POINTER(C.c_double)]
        L.ob_set_history.argtypes = [C.c_void_p, C.c_int, _dp, C.c_double, _dp, C.c_double,
                                     _dp, C.c_double, _dp, C.c_double]
        L.ob_spread_only.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _dp, C.POINTER(C.c_double)]
        L.ob_rigid_update.argtypes = [C.c_void_p, C.c_int, _dp, C.c_double]
        L.ob_set_threads.restype = C.c_int
        L.ob_set_threads.argtypes = [C.c_int]
        # one thread unless asked otherwise (many oracle processes may run
        # side by side)
        L.ob_set_threads(int(os.environ.get("OB_THREADS", "1")))
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's lattice loops; returns the count in use."""
    return lib().ob_set_threads(n)


# ---- single-step functions -------------------------------------------------

def lattice():
    e = np.zeros((9, 2), np.int32)
    w = np.zeros(9)
    lib().ob_lattice(e, w)
    return e, w


def feq(rho, ux, uy):
    out = np.zeros(9)
    lib().ob_feq(rho, ux, uy, out)
    return out


def collide(f, tau, Fx=0.0, Fy=0.0):
    out = np.zeros(9)
    lib().ob_collide(np.ascontiguousarray(f, np.float64), tau, Fx, Fy, out)
    return out


def guo_term(ux, uy, tau, Fx, Fy):
    out = np.zeros(9)
    lib().ob_guo_term(ux, uy, tau, Fx, Fy, out)
    return out


def mls(x, y, weight=W_EXP):
    ix = np.zeros(9, np.int32)
    iy = np.zeros(9, np.int32)
    phi = np.zeros(27)
    rc = lib().ob_mls(weight, x, y, ix, iy, phi)
    if rc != OK:
        raise RuntimeError("oracle MLS failed")
    return ix, iy, phi.reshape(3, 9)


def weight(kind, r):
    return lib().ob_weight(kind, r)


# ---- simulation ------------------------------------------------------------

class Sim:
    """One oracle lattice with its particles (FP64, CPU)."""

    def __init__(self, nx, ny, tau, bc=(PERIODIC, PERIODIC, VELOCITY, VELOCITY),
                 wall_u=((0, 0), (0, 0), (0, 0), (0, 0)), body_force=(0, 0), gravity=(0, 0),
                 init=INIT_REST, init_u=0.0, weight=W_EXP, spacing=0.3):
        c = Config()
        c.nx, c.ny, c.tau = nx, ny, tau
        for i in range(4):
            c.bc[i] = bc[i]
            c.wall_u[i][0], c.wall_u[i][1] = wall_u[i]
        c.body_force[0], c.body_force[1] = body_force
        c.gravity[0], c.gravity[1] = gravity
        c.init, c.init_u, c.weight, c.spacing = init, init_u, weight, spacing
        err = C.c_int(0)
        self._h = lib().ob_create(C.byref(c), C.byref(err))
        if not self._h:
            raise ValueError(f"oracle rejected the configuration (code {err.value})")
        self.nx, self.ny, self.tau = nx, ny, tau
        self.np = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ob_destroy(h)
            self._h = None

    def add_particle(self, shape, dim, xc, yc, theta=0.0, rho_s=1.0, u0=(0.0, 0.0), omega0=0.0,
                     n_markers=0):
        d = ParticleDesc()
        d.shape = shape
        d.dim[0] = dim[0]
        d.dim[1] = dim[1] if len(dim) > 1 else 0.0
        d.xc, d.yc, d.theta, d.rho_s = xc, yc, theta, rho_s
        d.u0[0], d.u0[1] = u0
        d.omega0, d.n_markers = omega0, n_markers
        rc = lib().ob_add_particle(self._h, C.byref(d))
        if rc != OK:
            raise ValueError(f"oracle rejected the particle: {self.last_error()}")
        self.np += 1
        return self.np - 1

    def last_error(self):
        return lib().ob_last_error(self._h).decode()

    def step(self, n=1):
        rc = lib().ob_step(self._h, n)
        if rc != OK:
            raise RuntimeError(f"oracle step failed ({rc}): {self.last_error()}")

    @property
    def steps_done(self):
        return lib().ob_steps_done(self._h)

    def populations(self):
        f = np.zeros(9 * self.nx * self.ny)
        lib().ob_get_populations(self._h, f)
        return f.reshape(9, self.ny, self.nx)

    def set_populations(self, f):
        lib().ob_set_populations(self._h, np.ascontiguousarray(f, np.float64).ravel())

    def fields(self):
        r = np.zeros(self.nx * self.ny)
        ux = np.zeros_like(r)
        uy = np.zeros_like(r)
        lib().ob_get_fields(self._h, r, ux, uy)
        sh = (self.ny, self.nx)
        return r.reshape(sh), ux.reshape(sh), uy.reshape(sh)

    def particles(self):
        arr = (ParticleState * max(self.np, 1))()
        lib().ob_get_particles(self._h, arr, self.np)
        out = []
        for i in range(self.np):
            p = arr[i]
            out.append(dict(xc=p.xc, yc=p.yc, theta=p.theta, u=(p.u[0], p.u[1]),
                            omega=p.omega, F=(p.F[0], p.F[1]), M=p.M))
        return out

    def markers(self, p):
        cap = 100000
        rb = np.zeros(2 * cap)
        nb = np.zeros(2 * cap)
        S = np.zeros(cap)
        n = lib().ob_get_markers(self._h, p, rb, nb, S, cap)
        return rb[: 2 * n].reshape(n, 2), nb[: 2 * n].reshape(n, 2), S[:n]

    def props(self, p):
        m, I, A = C.c_double(), C.c_double(), C.c_double()
        lib().ob_particle_props(self._h, p, C.byref(m), C.byref(I), C.byref(A))
        return m.value, I.value, A.value

    def force_field(self):
        f = np.zeros(2 * self.nx * self.ny)
        lib().ob_get_force_field(self._h, f)
        return f.reshape(2, self.ny, self.nx)

    def stress_force(self, p, rho, ux, uy):
        F = np.zeros(2)
        M = C.c_double()
        rc = lib().ob_stress_force(self._h, p, np.ascontiguousarray(rho, np.float64).ravel(),
                                   np.ascontiguousarray(ux, np.float64).ravel(),
                                   np.ascontiguousarray(uy, np.float64).ravel(), F, C.byref(M))
        if rc != OK:
            raise RuntimeError(f"stress force failed ({rc}): {self.last_error()}")
        return F, M.value

    def set_history(self, p, X1, th1, U1, W1, X2, th2, U2, W2):
        a = lambda v: np.ascontiguousarray(v, np.float64)
        lib().ob_set_history(self._h, p, a(X1), th1, a(U1), W1, a(X2), th2, a(U2), W2)

    def spread(self, p, ux, uy):
        flb = np.zeros(2 * self.nx * self.ny)
        sf = np.zeros(2)
        tq = C.c_double()
        rc = lib().ob_spread_only(self._h, p, np.ascontiguousarray(ux, np.float64).ravel(),
                                  np.ascontiguousarray(uy, np.float64).ravel(), flb, sf,
                                  C.byref(tq))
        if rc != OK:
            raise RuntimeError(f"spread failed ({rc}): {self.last_error()}")
        return flb.reshape(2, self.ny, self.nx), sf, tq.value

    def rigid_update(self, p, F, M):
        lib().ob_rigid_update(self._h, p, np.ascontiguousarray(F, np.float64), M)
