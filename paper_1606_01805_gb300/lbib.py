"""ctypes binding of the C ABI in ``include/lbib.h`` (liblbib.so).

Argument marshalling only: every stage of the LB-IB step runs in the CUDA
kernels of the library.  PyTorch supplies the device workspace (through its
caching allocator) and the CUDA stream.  Importing this module does not need
a GPU; creating a :class:`Simulation` does, and fails loudly if the library
has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

import numpy as np

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "liblbib.so"

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ETIMEOUT, LBM_ENONFINITE, LBM_EINTERNAL, LBM_EDOMAIN = range(8)
STATUS_NAMES = ["LBM_OK", "LBM_EINVAL", "LBM_ENOMEM", "LBM_ECUDA", "LBM_ETIMEOUT",
                "LBM_ENONFINITE", "LBM_EINTERNAL", "LBM_EDOMAIN"]
LBM_BC_PERIODIC, LBM_BC_VELOCITY = 0, 1
LBM_FP64, LBM_FP32, LBM_FP16_SHIFTED, LBM_FP32_TANGENT = 0, 1, 2, 3
LBM_TANGENTS = 3            # derivative directions of the tangent mode
LBM_TILE_VARIANTS = 10      # fluid tile variants (lbm_get_tile / lbm_set_tile / lbm_tile_info)
LBM_TANGENT_FIELDS = 10     # xc, yc, theta, u[0], u[1], omega, F[0], F[1], M, omega_sum
TANGENT_FIELDS = ("xc", "yc", "theta", "ux", "uy", "omega", "Fx", "Fy", "M", "omega_sum")
SEED_FIELDS = ("dim0", "dim1", "xc", "yc", "theta", "rho_s")
LBM_INIT_REST, LBM_INIT_COUETTE, LBM_INIT_TAYLOR_GREEN = 0, 1, 2
LBM_STEP_SEPARATE, LBM_STEP_FUSED, LBM_STEP_OVERLAP = 0, 1, 2  # step modes of a batch (lbm_set_step_mode)
LBM_SHAPE_CIRCLE, LBM_SHAPE_ELLIPSE, LBM_SHAPE_RECT, LBM_SHAPE_SQUARE, LBM_SHAPE_TRIANGLE = range(5)
LBM_W_EXP, LBM_W_CUBIC, LBM_W_QUARTIC, LBM_W_COSINE, LBM_W_POLY = range(5)

# every symbol include/lbib.h declares
EXPORTS = ["lbm_workspace_bytes", "lbm_init", "lbm_add_particle", "lbm_step", "lbm_step_timed",
           "lbm_sync", "lbm_inject_status", "lbm_inject_stall", "lbm_tile_info", "lbm_set_step_mode",
           "lbm_get_step_mode", "lbm_adjoint", "lbm_get_fields", "lbm_get_populations", "lbm_set_populations",
           "lbm_get_particles", "lbm_steps_done", "lbm_last_error", "lbm_destroy",
           "lbm_step_static", "lbm_batch_workspace_bytes", "lbm_init_batch", "lbm_instances",
           "lbm_add_particle_to", "lbm_get_instance_fields", "lbm_get_instance_populations",
           "lbm_set_instance_populations", "lbm_get_tile", "lbm_set_tile",
           "lbm_set_wall_tangents", "lbm_add_particle_tangent", "lbm_get_particle_tangents",
           "lbm_get_field_tangents"]
LBM_STATIC_MAX_PARTICLES, LBM_STATIC_MAX_MARKERS = 1024, 16384


class lbm_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("tau", C.c_double),
        ("bc", C.c_int32 * 4), ("wall_u", (C.c_double * 2) * 4),
        ("body_force", C.c_double * 2), ("gravity", C.c_double * 2),
        ("precision", C.c_int32), ("init", C.c_int32), ("init_u", C.c_double),
        ("weight", C.c_int32), ("marker_spacing", C.c_double),
        ("max_particles", C.c_int32), ("max_markers", C.c_int32),
        ("cuda_stream", C.c_void_p), ("d_workspace", C.c_void_p), ("workspace_bytes", C.c_size_t),
        ("check_every", C.c_int32),
    ]


class lbm_particle_desc(C.Structure):
    _fields_ = [
        ("shape", C.c_int32), ("dim", C.c_double * 2), ("xc", C.c_double), ("yc", C.c_double),
        ("theta", C.c_double), ("rho_s", C.c_double), ("u0", C.c_double * 2),
        ("omega0", C.c_double), ("n_markers", C.c_int32),
    ]


class lbm_particle_state(C.Structure):
    _fields_ = [
        ("xc", C.c_double), ("yc", C.c_double), ("theta", C.c_double), ("u", C.c_double * 2),
        ("omega", C.c_double), ("F", C.c_double * 2), ("M", C.c_double),
        ("omega_sum", C.c_double),
    ]


class LbmError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {what}")
        self.status = status


_lib = None
_dp = C.POINTER(C.c_double)


def load(path: os.PathLike | str | None = None):
    """Load liblbib.so (built by ``paper_1606_01805_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"{p} is missing: build it with `python -m paper_1606_01805_gb300.build`")
    L = C.CDLL(str(p))
    L.lbm_workspace_bytes.argtypes = [C.POINTER(lbm_config), C.POINTER(C.c_size_t)]
    L.lbm_init.argtypes = [C.POINTER(lbm_config), C.POINTER(C.c_void_p)]
    L.lbm_add_particle.argtypes = [C.c_void_p, C.POINTER(lbm_particle_desc), C.POINTER(C.c_int32)]
    L.lbm_step.argtypes = [C.c_void_p, C.c_int32]
    L.lbm_step_timed.argtypes = [C.c_void_p, C.c_int32, _dp, _dp]
    L.lbm_sync.argtypes = [C.c_void_p]
    L.lbm_inject_status.argtypes = [C.c_void_p, C.c_int32]
    L.lbm_inject_stall.argtypes = [C.c_void_p, C.c_int64]
    L.lbm_tile_info.argtypes = [C.c_int32, C.c_int32] + [C.POINTER(C.c_int32)] * 3
    L.lbm_set_step_mode.argtypes = [C.c_void_p, C.c_int32]
    L.lbm_adjoint.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _dp, _dp, _dp]
    L.lbm_get_step_mode.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    L.lbm_get_fields.argtypes = [C.c_void_p, _dp, _dp, _dp]
    L.lbm_get_populations.argtypes = [C.c_void_p, _dp]
    L.lbm_set_populations.argtypes = [C.c_void_p, _dp]
    L.lbm_get_particles.argtypes = [C.c_void_p, C.POINTER(lbm_particle_state), C.c_int32,
                                    C.POINTER(C.c_int32)]
    L.lbm_steps_done.restype = C.c_int64
    L.lbm_steps_done.argtypes = [C.c_void_p]
    L.lbm_last_error.restype = C.c_char_p
    L.lbm_last_error.argtypes = [C.c_void_p]
    L.lbm_destroy.argtypes = [C.c_void_p]
    L.lbm_destroy.restype = None
    L.lbm_step_static.argtypes = [C.c_void_p, C.c_int32]
    L.lbm_batch_workspace_bytes.argtypes = [C.POINTER(lbm_config), C.c_int32, C.POINTER(C.c_size_t)]
    L.lbm_init_batch.argtypes = [C.POINTER(lbm_config), C.c_int32, C.POINTER(C.c_void_p)]
    L.lbm_instances.restype = C.c_int32
    L.lbm_instances.argtypes = [C.c_void_p]
    L.lbm_add_particle_to.argtypes = [C.c_void_p, C.c_int32, C.POINTER(lbm_particle_desc),
                                      C.POINTER(C.c_int32)]
    L.lbm_get_instance_fields.argtypes = [C.c_void_p, C.c_int32, _dp, _dp, _dp]
    L.lbm_get_instance_populations.argtypes = [C.c_void_p, C.c_int32, _dp]
    L.lbm_set_instance_populations.argtypes = [C.c_void_p, C.c_int32, _dp]
    L.lbm_get_tile.argtypes = [C.c_void_p] + [C.POINTER(C.c_int32)] * 3
    L.lbm_set_tile.argtypes = [C.c_void_p, C.c_int32]
    L.lbm_set_wall_tangents.argtypes = [C.c_void_p, C.c_int32, _dp]
    L.lbm_add_particle_tangent.argtypes = [C.c_void_p, C.c_int32, C.POINTER(lbm_particle_desc), _dp,
                                           C.POINTER(C.c_int32)]
    L.lbm_get_particle_tangents.argtypes = [C.c_void_p, _dp, C.c_int32, C.POINTER(C.c_int32)]
    L.lbm_get_field_tangents.argtypes = [C.c_void_p, C.c_int32, _dp, _dp, _dp]
    for fn in ("lbm_workspace_bytes", "lbm_init", "lbm_add_particle", "lbm_step", "lbm_step_timed",
               "lbm_sync", "lbm_inject_status", "lbm_inject_stall", "lbm_tile_info", "lbm_set_step_mode",
               "lbm_get_step_mode", "lbm_adjoint", "lbm_get_fields", "lbm_get_populations", "lbm_set_populations",
               "lbm_get_particles", "lbm_step_static", "lbm_batch_workspace_bytes",
               "lbm_init_batch", "lbm_add_particle_to", "lbm_get_instance_fields",
               "lbm_get_instance_populations", "lbm_set_instance_populations", "lbm_get_tile",
               "lbm_set_tile", "lbm_set_wall_tangents", "lbm_add_particle_tangent",
               "lbm_get_particle_tangents", "lbm_get_field_tangents"):
        getattr(L, fn).restype = C.c_int
    _lib = L
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def make_config(nx, ny, tau, bc=(0, 0, 1, 1), wall_u=((0, 0),) * 4, body_force=(0, 0),
                gravity=(0, 0), precision=LBM_FP32, init=LBM_INIT_REST, init_u=0.0,
                weight=LBM_W_EXP, marker_spacing=0.3, max_particles=16, max_markers=16384,
                check_every=1):
    c = lbm_config()
    c.nx, c.ny, c.tau = nx, ny, tau
    for i in range(4):
        c.bc[i] = bc[i]
        c.wall_u[i][0], c.wall_u[i][1] = wall_u[i]
    c.body_force[0], c.body_force[1] = body_force
    c.gravity[0], c.gravity[1] = gravity
    c.precision, c.init, c.init_u = precision, init, init_u
    c.weight, c.marker_spacing = weight, marker_spacing
    c.max_particles, c.max_markers = max_particles, max_markers
    c.check_every = check_every
    return c


class Simulation:
    """One LB-IB lattice on the current CUDA device.

    The device workspace is a torch uint8 tensor; the stream is torch's
    current stream (or the one given)."""

    def __init__(self, nx, ny, tau, stream=None, **kw):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        L = load()
        self.cfg = make_config(nx, ny, tau, **kw)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.cfg.cuda_stream = C.c_void_p(self.stream.cuda_stream)
        nbytes = C.c_size_t()
        self._check(L.lbm_workspace_bytes(C.byref(self.cfg), C.byref(nbytes)), "workspace size")
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
        self.cfg.d_workspace = C.c_void_p(self.workspace.data_ptr())
        self.cfg.workspace_bytes = nbytes.value
        h = C.c_void_p()
        self._check(L.lbm_init(C.byref(self.cfg), C.byref(h)), "lbm_init")
        self._h = h
        self.nx, self.ny = nx, ny
        self.np = 0

    def _check(self, rc, what):
        if rc != LBM_OK:
            msg = load().lbm_last_error(self._h).decode() if getattr(self, "_h", None) else what
            raise LbmError(rc, msg or what)

    def close(self):
        if getattr(self, "_h", None):
            load().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_particle(self, shape, dim, xc, yc, theta=0.0, rho_s=1.0, u0=(0.0, 0.0), omega0=0.0,
                     n_markers=0, tangent=None):
        """Add a particle; `tangent` (tangent mode only) is an array
        [LBM_TANGENTS][6] of d(dim0, dim1, xc, yc, theta, rho_s)/dp_k."""
        return _add(self, 0, shape, dim, xc, yc, theta, rho_s, u0, omega0, n_markers, tangent)

    def step(self, n=1):
        self._check(load().lbm_step(self._h, n), "lbm_step")

    def step_timed(self, n=1, fluid=True):
        """(ms of the n steps, ms of their fluid kernels); fluid=False leaves
        out the event before the fluid kernel (see lbm_step_timed) and
        returns 0 for the second figure."""
        ms_step, ms_fluid = C.c_double(0), C.c_double(0)
        self._check(load().lbm_step_timed(self._h, n, C.byref(ms_step),
                                          C.byref(ms_fluid) if fluid else None), "lbm_step_timed")
        return ms_step.value, ms_fluid.value

    def sync(self):
        self._check(load().lbm_sync(self._h), "lbm_sync")

    def inject_status(self, status):
        """Test hook: the device flag of `status`, as a kernel sets it."""
        self._check(load().lbm_inject_status(self._h, status), "lbm_inject_status")

    def inject_stall(self, wait_cycles):
        """Test hook: the next step's staged fluid launch waits for a copy
        that never comes, for wait_cycles clock cycles (lbm_inject_stall)."""
        self._check(load().lbm_inject_stall(self._h, wait_cycles), "lbm_inject_stall")

    @property
    def steps_done(self):
        return load().lbm_steps_done(self._h)

    def fields(self, out=None):
        """(rho, ux, uy) as [ny][nx] arrays; `out`: three caller arrays
        (C-contiguous float64, e.g. in pinned memory) to fill instead."""
        r, ux, uy = out if out is not None else [np.empty((self.ny, self.nx)) for _ in range(3)]
        for a in (r, ux, uy):
            assert a.dtype == np.float64 and a.shape == (self.ny, self.nx) and a.flags.c_contiguous
        self._check(load().lbm_get_fields(self._h, _ptr(r), _ptr(ux), _ptr(uy)), "lbm_get_fields")
        return r, ux, uy

    def populations(self, out=None):
        """stored populations [9][ny][nx]; `out`: a caller array to fill"""
        f = out if out is not None else np.empty((9, self.ny, self.nx))
        assert f.dtype == np.float64 and f.shape == (9, self.ny, self.nx) and f.flags.c_contiguous
        self._check(load().lbm_get_populations(self._h, _ptr(f)), "lbm_get_populations")
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, np.float64)
        assert f.shape == (9, self.ny, self.nx)
        self._check(load().lbm_set_populations(self._h, _ptr(f)), "lbm_set_populations")

    def particles(self):
        n = max(self.np, 1)
        arr = (lbm_particle_state * n)()
        cnt = C.c_int32()
        self._check(load().lbm_get_particles(self._h, arr, n, C.byref(cnt)), "lbm_get_particles")
        return [dict(xc=p.xc, yc=p.yc, theta=p.theta, u=(p.u[0], p.u[1]), omega=p.omega,
                     F=(p.F[0], p.F[1]), M=p.M, omega_sum=p.omega_sum) for p in arr[: cnt.value]]

    def particle_tangents(self):
        """Tangent mode: [particles][LBM_TANGENTS][LBM_TANGENT_FIELDS] array of
        d(state)/dp_k, fields in TANGENT_FIELDS order."""
        n = max(self.np, 1)
        out = np.zeros((n, LBM_TANGENTS, LBM_TANGENT_FIELDS))
        cnt = C.c_int32()
        self._check(load().lbm_get_particle_tangents(self._h, _ptr(out), n, C.byref(cnt)),
                    "lbm_get_particle_tangents")
        return out[: cnt.value]

    def set_wall_tangents(self, dwall, instance=0):
        """Tangent mode: dwall[side][c][k] = d(wall_u[side][c])/dp_k."""
        dw = np.ascontiguousarray(dwall, np.float64).reshape(4, 2, LBM_TANGENTS)
        self._check(load().lbm_set_wall_tangents(self._h, instance, _ptr(dw)), "lbm_set_wall_tangents")

    def field_tangents(self, instance=0):
        """Tangent mode: d(rho, ux, uy)/dp_k as three [LBM_TANGENTS][ny][nx] arrays."""
        ny, nx = self._shape(instance)
        out = [np.empty((LBM_TANGENTS, ny, nx)) for _ in range(3)]
        self._check(load().lbm_get_field_tangents(self._h, instance, *(_ptr(a) for a in out)),
                    "lbm_get_field_tangents")
        return tuple(out)

    def _shape(self, instance):
        return (self.ny, self.nx)

    def adjoint(self, nsteps, checkpoint_every, seed):
        """Reverse-mode gradients (lbm_adjoint): runs nsteps forward, then
        back; seed [np][2] weights the particles' final y and omega sum in
        the two outputs.  Returns (dparticle [np][2][6] over (dim0, dim1,
        xc, yc, theta, rho_s), dwall [instances][2][8] over wall_u[4][2])."""
        n = max(self.np, 1)
        seed = np.ascontiguousarray(seed, np.float64).reshape(n, 2)
        dp = np.zeros((n, 2, 6))
        dw = np.zeros((len(self) if isinstance(self, Batch) else 1, 2, 8))
        self._check(load().lbm_adjoint(self._h, nsteps, checkpoint_every, _ptr(seed), _ptr(dp), _ptr(dw)),
                    "lbm_adjoint")
        return dp, dw


class Batch:
    """Many independent lattices advanced together (lbm_init_batch).

    `configs` is a list of dicts of make_config keyword arguments (nx, ny,
    tau, bc, wall_u, ...); the first one also gives precision, weight and
    the batch-wide capacities."""

    def __init__(self, configs, stream=None, max_particles=None, max_markers=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        L = load()
        n = len(configs)
        arr = (lbm_config * n)()
        for i, kw in enumerate(configs):
            kw = dict(kw)
            nx, ny, tau = kw.pop("nx"), kw.pop("ny"), kw.pop("tau")
            arr[i] = make_config(nx, ny, tau, **kw)
        if max_particles is not None:
            arr[0].max_particles = max_particles
        if max_markers is not None:
            arr[0].max_markers = max_markers
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr[0].cuda_stream = C.c_void_p(self.stream.cuda_stream)
        nbytes = C.c_size_t()
        rc = L.lbm_batch_workspace_bytes(arr, n, C.byref(nbytes))
        if rc != LBM_OK:
            raise LbmError(rc, "batch workspace size")
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
        arr[0].d_workspace = C.c_void_p(self.workspace.data_ptr())
        arr[0].workspace_bytes = nbytes.value
        self._cfgs = arr
        h = C.c_void_p()
        rc = L.lbm_init_batch(arr, n, C.byref(h))
        if rc != LBM_OK:
            raise LbmError(rc, "lbm_init_batch")
        self._h = h
        self.shapes = [(c["ny"], c["nx"]) for c in configs]
        self.np = 0

    _check = Simulation._check
    close = Simulation.close
    __del__ = Simulation.__del__
    step = Simulation.step
    step_timed = Simulation.step_timed
    sync = Simulation.sync
    inject_status = Simulation.inject_status
    inject_stall = Simulation.inject_stall
    particles = Simulation.particles
    steps_done = Simulation.steps_done

    def __len__(self):
        return load().lbm_instances(self._h)

    particle_tangents = Simulation.particle_tangents
    adjoint = Simulation.adjoint
    set_wall_tangents = Simulation.set_wall_tangents
    field_tangents = Simulation.field_tangents

    def _shape(self, instance):
        return self.shapes[instance]

    def set_step_mode(self, mode):
        """LBM_STEP_SEPARATE, LBM_STEP_OVERLAP (two halves of the instances on two
        streams) or LBM_STEP_FUSED (one persistent launch per step)."""
        self._check(load().lbm_set_step_mode(self._h, mode), "lbm_set_step_mode")

    def step_mode(self):
        m = C.c_int32()
        self._check(load().lbm_get_step_mode(self._h, C.byref(m)), "lbm_get_step_mode")
        return m.value

    def add_particle(self, instance, shape, dim, xc, yc, theta=0.0, rho_s=1.0, u0=(0.0, 0.0),
                     omega0=0.0, n_markers=0, tangent=None):
        return _add(self, instance, shape, dim, xc, yc, theta, rho_s, u0, omega0, n_markers, tangent)

    def fields(self, instance):
        ny, nx = self.shapes[instance]
        r = np.empty((ny, nx))
        ux = np.empty_like(r)
        uy = np.empty_like(r)
        self._check(load().lbm_get_instance_fields(self._h, instance, _ptr(r), _ptr(ux), _ptr(uy)),
                    "lbm_get_instance_fields")
        return r, ux, uy

    def populations(self, instance):
        ny, nx = self.shapes[instance]
        f = np.empty((9, ny, nx))
        self._check(load().lbm_get_instance_populations(self._h, instance, _ptr(f)),
                    "lbm_get_instance_populations")
        return f

    def set_populations(self, instance, f):
        ny, nx = self.shapes[instance]
        f = np.ascontiguousarray(f, np.float64)
        assert f.shape == (9, ny, nx)
        self._check(load().lbm_set_instance_populations(self._h, instance, _ptr(f)),
                    "lbm_set_instance_populations")

    tile = None  # set below
    set_tile = None


def _add(obj, instance, shape, dim, xc, yc, theta, rho_s, u0, omega0, n_markers, tangent):
    d = lbm_particle_desc()
    d.shape = shape
    d.dim[0] = dim[0]
    d.dim[1] = dim[1] if len(dim) > 1 else 0.0
    d.xc, d.yc, d.theta, d.rho_s = xc, yc, theta, rho_s
    d.u0[0], d.u0[1] = u0
    d.omega0, d.n_markers = omega0, n_markers
    pid = C.c_int32()
    L = load()
    if tangent is not None:
        seed = np.ascontiguousarray(tangent, np.float64).reshape(LBM_TANGENTS, len(SEED_FIELDS))
        rc = L.lbm_add_particle_tangent(obj._h, instance, C.byref(d), _ptr(seed), C.byref(pid))
    else:
        rc = L.lbm_add_particle_to(obj._h, instance, C.byref(d), C.byref(pid))
    obj._check(rc, "lbm_add_particle")
    obj.np += 1
    return pid.value


def _tile(self):
    v, c, b = C.c_int32(), C.c_int32(), C.c_int32()
    self._check(load().lbm_get_tile(self._h, C.byref(v), C.byref(c), C.byref(b)), "lbm_get_tile")
    return v.value, c.value, b.value


def tile_info(variant, precision):
    """(cells per thread, rows per tile, stages, available) of a tile variant
    for a precision (lbm_tile_info)."""
    c, r, s = C.c_int32(), C.c_int32(), C.c_int32()
    rc = load().lbm_tile_info(variant, precision, C.byref(c), C.byref(r), C.byref(s))
    return c.value, r.value, s.value, rc == LBM_OK


def _set_tile(self, variant):
    self._check(load().lbm_set_tile(self._h, variant), "lbm_set_tile")


Simulation.tile = _tile
Simulation.set_tile = _set_tile
Batch.tile = _tile
Batch.set_tile = _set_tile
