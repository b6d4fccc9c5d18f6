"""FP64 CPU oracle for the tracer-box lattice Boltzmann method (arXiv:0809.4958).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the product library never imports it.
The arithmetic lives in ``lboracle.c`` (plain C, FP64, site by site); this
module compiles it with gcc and marshals numpy arrays.

Array layouts (all C-contiguous float64 unless stated):
  populations f      [19][E][E][E]   (index i, z, y, x; x fastest)
  velocity field u   [3][E][E][E]
  coarse samples     [J][6][3][E][E] (sample j at t = j K; face order x-, x+,
                                      y-, y+, z-, z+; in-face (q, p) = (z, y)
                                      on x faces, (z, x) on y faces, (y, x) on
                                      z faces)
  MLP residuals      [Jint][6][3][K][E][E]
  bead pos / vel     [N][3]

Parity pins for every function are in tests/test_oracle_*.py.  Parity
unpinned: none of the functions here; the turbulent-boundary runs themselves
have no closed form and are compared only against the GPU path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lboracle.c")
_LIB = os.path.join(_HERE, "liblboracle.so")

Q = 19
OK, ERR_ARG, ERR_FENE, ERR_BEAD_OOB, ERR_SAMPLES = 0, 1, 2, 3, 4
TIME_LINEAR, TIME_HERMITE, TIME_MLP = 0, 1, 2
STORE_F64, STORE_F16, STORE_BF16 = 0, 2, 3


def build(force: bool = False) -> str:
    """Compile lboracle.c into liblboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Box(ctypes.Structure):
    _fields_ = [
        ("E", ctypes.c_int32),
        ("periodic", ctypes.c_int32 * 3),
        ("tau", ctypes.c_double),
        ("rho_b", ctypes.c_double),
        ("accel", ctypes.c_double * 3),
        ("time_interp", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("zoom", ctypes.c_int32),
    ]


class _Chain(ctypes.Structure):
    _fields_ = [
        ("nbeads", ctypes.c_int32),
        ("n_md", ctypes.c_int32),
        ("pin_com", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("k_fene", ctypes.c_double),
        ("R0", ctypes.c_double),
        ("zeta", ctypes.c_double),
        ("mass", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("f_ext", ctypes.c_double * 3),
        ("seed", ctypes.c_uint64),
        ("box_id", ctypes.c_uint64),
    ]


_lib = None
_P = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_step.restype = ctypes.c_int
        lib.orc_run.restype = ctypes.c_int
        lib.orc_chain_couple.restype = ctypes.c_int
        lib.orc_chain_forces.restype = ctypes.c_int
        lib.orc_interp_velocity.restype = ctypes.c_int
        lib.orc_face_velocity.restype = ctypes.c_int
        lib.orc_round_f16.restype = ctypes.c_double
        lib.orc_round_f16.argtypes = [ctypes.c_double]
        lib.orc_round_bf16.restype = ctypes.c_double
        lib.orc_round_bf16.argtypes = [ctypes.c_double]
        lib.orc_equilibrium.argtypes = [ctypes.c_double, _P, _P]
        lib.orc_num_threads.restype = ctypes.c_int
        for name in ("orc_run", "orc_step", "orc_face_velocity"):
            getattr(lib, name).argtypes = None
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class BoxParams:
    """One tracer box: E sites per axis, BGK tau, per-axis periodic flags
    (False = both faces carry the velocity condition), boundary density,
    body acceleration, time interpolation, steps per coarse sample K and the
    storage emulation (STORE_F64 / STORE_F16 / STORE_BF16)."""
    E: int
    tau: float
    periodic: tuple = (False, False, False)
    rho_b: float = 1.0
    accel: tuple = (0.0, 0.0, 0.0)
    time_interp: int = TIME_LINEAR
    K: int = 1
    storage: int = STORE_F64
    zoom: int = 1

    def coarse_points(self):
        """Points per axis of the coarse grid (samples and initial field)."""
        return coarse_points(self.E, self.zoom)

    def c(self):
        b = _Box()
        b.E = self.E
        for a in range(3):
            b.periodic[a] = 1 if self.periodic[a] else 0
            b.accel[a] = float(self.accel[a])
        b.tau = float(self.tau)
        b.rho_b = float(self.rho_b)
        b.time_interp = int(self.time_interp)
        b.K = int(self.K)
        b.storage = int(self.storage)
        b.zoom = int(self.zoom)
        return b


def coarse_points(E, zoom=1):
    """Points per axis of the coarse grid: point P at site P zoom, until the
    grid covers site E - 1 (every site for zoom 1)."""
    return (E - 1 + zoom - 1) // zoom + 1 if zoom > 1 else E


@dataclass
class ChainParams:
    """Kremer-Grest bead-spring chain (FENE bonds + WCA repulsion) coupled by
    Stokes friction; eps = 0 leaves FENE bonds only."""
    nbeads: int
    k_fene: float = 30.0
    R0: float = 1.5
    zeta: float = 1.0
    mass: float = 1.0
    kT: float = 0.0
    eps: float = 1.0
    sigma: float = 1.0
    seed: int = 0
    n_md: int = 50
    pin_com: int = 2
    f_ext: tuple = (0.0, 0.0, 0.0)
    box_id: int = 0

    def c(self):
        ch = _Chain()
        ch.nbeads = self.nbeads
        ch.n_md = self.n_md
        ch.pin_com = self.pin_com
        ch.k_fene, ch.R0, ch.zeta, ch.mass, ch.kT = self.k_fene, self.R0, self.zeta, self.mass, self.kT
        ch.eps, ch.sigma = self.eps, self.sigma
        for a in range(3):
            ch.f_ext[a] = float(self.f_ext[a])
        ch.seed = int(self.seed) & 0xFFFFFFFFFFFFFFFF
        ch.box_id = int(self.box_id) & 0xFFFFFFFFFFFFFFFF
        return ch


def lattice():
    """D3Q19 velocities c [19][3] (int) and weights w [19]."""
    lib = _load()
    c = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q)
    lib.orc_lattice(_ptr(c), _ptr(w))
    return c.astype(np.int64), w


def equilibrium(rho, u):
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(Q)
    lib.orc_equilibrium(float(rho), u.ctypes.data_as(_P), out.ctypes.data_as(_P))
    return out


def round_f16(x: float) -> float:
    return _load().orc_round_f16(float(x))


def round_bf16(x: float) -> float:
    return _load().orc_round_bf16(float(x))


def philox4x32_10(ctr, key):
    """Philox4x32-10 of a 4-word counter and a 2-word key (uint32 words)."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def chain_forces(pos, k, R0, eps=1.0, sigma=1.0):
    """(status, F [N][3]) of the FENE + WCA chain at positions pos [N][3]."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    F = np.zeros_like(pos)
    st = lib.orc_chain_forces(ctypes.c_int(pos.shape[0]), ctypes.c_double(k), ctypes.c_double(R0),
                              ctypes.c_double(eps), ctypes.c_double(sigma), _ptr(pos), _ptr(F))
    return st, F


def init(box: BoxParams, u0):
    """Initial condition: equilibrium with rho = 1 and the velocity u0 given on
    the coarse grid [3][Ec^3] (every site when zoom = 1), trilinear in between."""
    lib = _load()
    E, Ec = box.E, box.coarse_points()
    u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape(3, Ec, Ec, Ec)
    f = np.zeros((Q, E, E, E))
    b = box.c()
    lib.orc_init(ctypes.byref(b), _ptr(u0), _ptr(f))
    return f


class Sim:
    """Oracle state of one box: populations f (post-collision, step n) plus an
    optional chain.  ``run(k)`` advances k steps."""

    def __init__(self, box: BoxParams, u0, samples, chain: ChainParams | None = None,
                 pos0=None, vel0=None, resid=None, n0: int = 0):
        self.box = box
        self.E = box.E
        self.f = init(box, u0)
        self.tmp = np.zeros_like(self.f)
        self.g = np.zeros((3,) + self.f.shape[1:])
        self.samples = np.ascontiguousarray(samples, dtype=np.float64)
        self.resid = None if resid is None else np.ascontiguousarray(resid, dtype=np.float64)
        self.chain = chain
        if chain is not None:
            self.pos = np.ascontiguousarray(pos0, dtype=np.float64).copy()
            self.vel = (np.zeros_like(self.pos) if vel0 is None
                        else np.ascontiguousarray(vel0, dtype=np.float64).copy())
        else:
            self.pos = np.zeros((0, 3))
            self.vel = np.zeros((0, 3))
        self.n = n0

    def run(self, nsteps: int) -> int:
        lib = _load()
        b = self.box.c()
        ch = self.chain.c() if self.chain is not None else None
        st = lib.orc_run(
            ctypes.byref(b), ctypes.byref(ch) if ch is not None else None,
            _ptr(self.f), _ptr(self.tmp), _ptr(self.g), _ptr(self.samples),
            ctypes.c_long(self.samples.shape[0]), _ptr(self.resid),
            ctypes.c_long(self.n), ctypes.c_long(nsteps), _ptr(self.pos), _ptr(self.vel))
        if st == 0:
            self.n += nsteps
        return st

    def fields(self):
        """(rho [E^3], u [3][E^3]) per the reported-field definition."""
        return fields(self.box, self.f)

    def conservation(self):
        return conservation(self.box, self.f, self.chain, self.vel)


def step_from(box: BoxParams, A, samples, n, chain: ChainParams | None = None, pos=None, vel=None,
              resid=None):
    """One step n -> n+1 from an arbitrary state A (e.g. one read back from
    the GPU).  Returns (status, B, pos, vel, g)."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.zeros_like(A)
    g = np.zeros((3,) + A.shape[1:])
    samples = np.ascontiguousarray(samples, dtype=np.float64)
    b = box.c()
    ch = chain.c() if chain is not None else None
    pos = None if pos is None else np.ascontiguousarray(pos, dtype=np.float64).copy()
    vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64).copy()
    st = lib.orc_step(ctypes.byref(b), ctypes.byref(ch) if ch is not None else None, _ptr(A), _ptr(B), _ptr(g),
                      _ptr(samples), ctypes.c_long(samples.shape[0]),
                      _ptr(None if resid is None else np.ascontiguousarray(resid, dtype=np.float64)),
                      ctypes.c_long(n), _ptr(pos), _ptr(vel))
    return st, B, pos, vel, g


def chain_couple(box: BoxParams, chain: ChainParams, A, n, pos, vel):
    """Bead coupling of step n alone: returns (status, pos, vel, g [3][E^3])."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    pos = np.ascontiguousarray(pos, dtype=np.float64).copy()
    vel = np.ascontiguousarray(vel, dtype=np.float64).copy()
    g = np.zeros((3,) + A.shape[1:])
    b = box.c()
    ch = chain.c()
    st = lib.orc_chain_couple(ctypes.byref(b), ctypes.byref(ch), _ptr(A), ctypes.c_long(n), _ptr(pos), _ptr(vel), _ptr(g))
    return st, pos, vel, g


def interp_velocity(box: BoxParams, A, R):
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    u = np.zeros(3)
    b = box.c()
    st = lib.orc_interp_velocity(ctypes.byref(b), _ptr(A), _ptr(R), _ptr(u))
    return st, u


def face_velocity(box: BoxParams, samples, n, f, p, q, resid=None):
    lib = _load()
    samples = np.ascontiguousarray(samples, dtype=np.float64)
    u = np.zeros(3)
    b = box.c()
    st = lib.orc_face_velocity(ctypes.byref(b), _ptr(samples), ctypes.c_long(samples.shape[0]),
                               _ptr(None if resid is None else np.ascontiguousarray(resid, dtype=np.float64)),
                               ctypes.c_long(n), ctypes.c_int(f), ctypes.c_int(p), ctypes.c_int(q), _ptr(u))
    return st, u


def fields(box: BoxParams, A):
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    E = box.E
    rho = np.zeros((E, E, E))
    u = np.zeros((3, E, E, E))
    b = box.c()
    lib.orc_fields(ctypes.byref(b), _ptr(A), _ptr(rho), _ptr(u))
    return rho, u


def conservation(box: BoxParams, A, chain: ChainParams | None = None, vel=None):
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.zeros(7)
    b = box.c()
    nb = 0 if chain is None else chain.nbeads
    mass = 1.0 if chain is None else chain.mass
    v = np.zeros((0, 3)) if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
    lib.orc_conservation(ctypes.byref(b), _ptr(A), ctypes.c_int(nb), ctypes.c_double(mass), _ptr(v), _ptr(out))
    return out


def field(modes, E, pts, t):
    """Synthetic coarse flow u(x, t) at points pts [n][3]."""
    lib = _load()
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.zeros_like(pts)
    xc = np.full(3, 0.5 * (E - 1))
    lib.orc_field(_ptr(modes.kvec), _ptr(modes.amp), _ptr(modes.omega), _ptr(modes.phi), ctypes.c_int(modes.M),
                  _ptr(xc), _ptr(pts), ctypes.c_long(pts.shape[0]), ctypes.c_double(t), _ptr(out))
    return out


def face_samples(modes, E, K, j0, nsamp, zoom=1):
    """Coarse face samples j0..j0+nsamp-1 at t = j K on the coarse face points
    (site P zoom): [nsamp][6][3][Ec][Ec], Ec = coarse_points(E, zoom)."""
    lib = _load()
    Ec = coarse_points(E, zoom)
    out = np.zeros((nsamp, 6, 3, Ec, Ec))
    lib.orc_face_samples(_ptr(modes.kvec), _ptr(modes.amp), _ptr(modes.omega), _ptr(modes.phi), ctypes.c_int(modes.M),
                         ctypes.c_int(E), ctypes.c_int(zoom), ctypes.c_int(K), ctypes.c_long(j0),
                         ctypes.c_long(nsamp), _ptr(out))
    return out


def volume_field(modes, E, t=0.0, zoom=1):
    """Synthetic flow at time t on the coarse grid (every zoom-th site; every
    site when zoom = 1): [3][Ec][Ec][Ec]."""
    lib = _load()
    Ec = coarse_points(E, zoom)
    out = np.zeros((3, Ec, Ec, Ec))
    lib.orc_volume_field(_ptr(modes.kvec), _ptr(modes.amp), _ptr(modes.omega), _ptr(modes.phi), ctypes.c_int(modes.M),
                         ctypes.c_int(E), ctypes.c_int(zoom), ctypes.c_double(t), _ptr(out))
    return out


def num_threads() -> int:
    return int(_load().orc_num_threads())


def vorticity_mean(u, lo, hi):
    """Mean magnitude of the vorticity over the cube lo <= x, y, z <= hi of a
    velocity field u [3][E][E][E] (layout [c][z][y][x]), omega = curl u by
    second-order central differences (Sec. 3, Figs. 1 and 2: |omega| averaged
    over the sub-volume around the tracer and over a region at its centre).
    The cube must lie inside sites 1 .. E-2.  FP64, numpy."""
    u = np.asarray(u, dtype=np.float64)
    E = u.shape[1]
    assert 1 <= lo <= hi <= E - 2
    c = slice(lo, hi + 1)
    p, m = slice(lo + 1, hi + 2), slice(lo - 1, hi)

    def d(comp, axis):  # central difference of u[comp] along axis (0 = z, 1 = y, 2 = x) on the cube
        a = [c, c, c]
        b = [c, c, c]
        a[axis], b[axis] = p, m
        return 0.5 * (u[comp][tuple(a)] - u[comp][tuple(b)])

    wx = d(2, 1) - d(1, 0)  # d u_z / dy - d u_y / dz
    wy = d(0, 0) - d(2, 2)  # d u_x / dz - d u_z / dx
    wz = d(1, 2) - d(0, 1)  # d u_y / dx - d u_x / dy
    return float(np.sqrt(wx * wx + wy * wy + wz * wz).mean())


def frame_accel_at(accel, frame_samples, K, n):
    """Body acceleration of step n of a box in the tracer's co-moving frame
    (Sec. 2: the transformed flow w = u - v(t) feels the force density
    rho (-dv/dt)): the constant body acceleration plus the frame-acceleration
    samples [J][3] (taken at t = jK) interpolated linearly at t_n between
    samples j = n // K and j + 1."""
    j = n // K
    th = (n - j * K) / K
    a = np.asarray(accel, dtype=np.float64) + (1.0 - th) * np.asarray(frame_samples[j], dtype=np.float64)
    return a + th * np.asarray(frame_samples[j + 1], dtype=np.float64)


def run_frame(box: BoxParams, A, samples, frame_samples, n0, nsteps, chain: ChainParams | None = None, pos=None,
              vel=None):
    """Steps n0 .. n0 + nsteps - 1 from state A with the body acceleration of
    each step taken from frame_accel_at (the box's own accel is the constant
    part).  Returns (status, A, pos, vel)."""
    from dataclasses import replace
    for n in range(n0, n0 + nsteps):
        bn = replace(box, accel=tuple(frame_accel_at(box.accel, frame_samples, box.K, n)))
        st, A, pos, vel, _ = step_from(bn, A, samples, n, chain, pos, vel)
        if st:
            return st, A, pos, vel
    return 0, A, pos, vel

