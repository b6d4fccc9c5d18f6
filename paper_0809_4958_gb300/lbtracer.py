"""Python binding of the C ABI in include/lbtracer.h (argument marshalling only).

Every function of the C ABI is exposed under the same name; the ``Tracers``
class bundles a context with its caller-owned device arena (a torch uint8
tensor) and the stream it runs on.  All arithmetic of the method runs in the
CUDA kernels of liblbtracer.so; there is no CPU path: loading fails loudly when
the library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LB_OK, LB_ERR_ARG, LB_ERR_CUDA, LB_ERR_FENE, LB_ERR_BEAD_OOB = 0, 1, 2, 3, 4
LB_ERR_NONFINITE, LB_ERR_TIMEOUT, LB_ERR_STATE, LB_ERR_SIZE, LB_ERR_CHAIN = 5, 6, 7, 8, 9
LB_STORE_F64, LB_STORE_F32, LB_STORE_F16DEV, LB_STORE_BF16DEV = 0, 1, 2, 3
LB_FACE_VELOCITY, LB_FACE_PERIODIC = 0, 1
LB_TIME_LINEAR, LB_TIME_HERMITE, LB_TIME_MLP = 0, 1, 2
LB_FIELD_RHO, LB_FIELD_U, LB_FIELD_DEV, LB_FIELD_CHAIN, LB_FIELD_ASYNC = 0, 1, 2, 3, 0x100
LB_ALL_BOXES = -1
LB_KERNEL_STAGED, LB_KERNEL_REGISTER = 0, 1
LB_INJECT_NONE, LB_INJECT_WITHHOLD_LAST_TILE = 0, 1

ERROR_NAMES = {0: "LB_OK", 1: "LB_ERR_ARG", 2: "LB_ERR_CUDA", 3: "LB_ERR_FENE", 4: "LB_ERR_BEAD_OOB",
               5: "LB_ERR_NONFINITE", 6: "LB_ERR_TIMEOUT", 7: "LB_ERR_STATE", 8: "LB_ERR_SIZE", 9: "LB_ERR_CHAIN"}

EXPORTS = ["lb_plan", "lb_create", "lb_destroy", "lb_init", "lb_set_boundary", "chain_couple", "lb_step",
           "lb_graph_capture", "lb_graph_launch", "lb_read_fields", "lb_conservation", "lb_checkpoint_bytes", "lb_save",
           "lb_load", "lb_vorticity", "lb_set_frame_accel", "lb_sync",
           "lb_status",
           "lb_current_step", "lb_set_launch", "lb_set_bead_launch", "lb_set_chain_history", "lb_set_fluctuation", "lb_test_inject", "lb_profile", "lb_profile_read", "lb_last_error", "lb_synth_workspace_bytes", "lb_synth_faces",
           "lb_synth_volume", "lb_population_sums_noalloc", "lb_mlp_param_bytes", "lb_mlp_bind", "lb_mlp_train_bytes",
           "lb_mlp_train_init", "lb_mlp_features", "lb_mlp_targets", "lb_mlp_forward", "lb_mlp_grad",
           "lb_mlp_train_step", "lb_mlp_export"]


class lb_box_desc(ctypes.Structure):
    _fields_ = [("E", ctypes.c_int32), ("face_mode", ctypes.c_int32 * 6), ("time_interp", ctypes.c_int32),
                ("K", ctypes.c_int32), ("nbeads", ctypes.c_int32), ("zoom", ctypes.c_int32),
                ("frame_accel", ctypes.c_int32), ("tau", ctypes.c_double), ("rho_b", ctypes.c_double),
                ("body_accel", ctypes.c_double * 3)]


class lb_chain_desc(ctypes.Structure):
    _fields_ = [("nbeads", ctypes.c_int32), ("n_md", ctypes.c_int32), ("pin_com", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("k_fene", ctypes.c_double), ("R0", ctypes.c_double),
                ("zeta", ctypes.c_double), ("mass", ctypes.c_double), ("kT", ctypes.c_double),
                ("eps", ctypes.c_double), ("sigma", ctypes.c_double), ("f_ext", ctypes.c_double * 3),
                ("seed", ctypes.c_uint64)]


class LBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (ERROR_NAMES.get(code, str(code)), msg))
        self.code = code


_lib = None
_vp, _i32, _i64, _f64, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t


def load(path: str | None = None, build_if_missing: bool = True):
    """Load liblbtracer.so (building it in place with nvcc if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise OSError("liblbtracer.so is not built (run paper_0809_4958_gb300/build.py)")
            _build.build()
    lib = ctypes.CDLL(path)
    sig = {
        "lb_plan": (_i32, [ctypes.POINTER(lb_box_desc), _i32, _i32, _i32, ctypes.POINTER(_sz)]),
        "lb_create": (_i32, [ctypes.POINTER(lb_box_desc), _i32, _i32, _i32, _vp, _sz, _vp, ctypes.POINTER(_vp)]),
        "lb_destroy": (_i32, [_vp]),
        "lb_init": (_i32, [_vp, _i32, _vp]),
        "lb_set_boundary": (_i32, [_vp, _i32, _i64, _vp]),
        "chain_couple": (_i32, [_vp, _i32, ctypes.POINTER(lb_chain_desc), _vp, _vp]),
        "lb_step": (_i32, [_vp, _i32]),
        "lb_graph_capture": (_i32, [_vp, _i32]),
        "lb_graph_launch": (_i32, [_vp]),
        "lb_read_fields": (_i32, [_vp, _i32, _i32, _vp]),
        "lb_conservation": (_i32, [_vp, _i32, _vp]),
        "lb_checkpoint_bytes": (_sz, [_vp]),
        "lb_save": (_i32, [_vp, _vp]),
        "lb_load": (_i32, [_vp, _vp]),
        "lb_vorticity": (_i32, [_vp, _i32, _i32, _i32, _vp]),
        "lb_set_frame_accel": (_i32, [_vp, _i32, _i64, _vp]),
        "lb_sync": (_i32, [_vp, _i32]),
        "lb_status": (_i32, [_vp, _i32, ctypes.POINTER(_i32)]),
        "lb_current_step": (_i64, [_vp]),
        "lb_set_launch": (_i32, [_vp, _i32, _i32, _i32, _i32]),
        "lb_set_bead_launch": (_i32, [_vp, _i32, _i32]),
        "lb_set_chain_history": (_i32, [_vp, _vp, _i32]),
        "lb_test_inject": (_i32, [_vp, _i32, _i32]),
        "lb_set_fluctuation": (_i32, [_vp, _i32, _f64, ctypes.c_uint64, _vp]),
        "lb_profile": (_i32, [_vp, _i32, _i32]),
        "lb_profile_read": (_i32, [_vp, ctypes.POINTER(_f64), ctypes.POINTER(_i64)]),
        "lb_last_error": (ctypes.c_char_p, [_vp]),
        "lb_synth_workspace_bytes": (_sz, [_i32, _i32]),
        "lb_synth_faces": (_i32, [_vp, _vp, _vp, _vp, _i32, _i32, _i32, _i32, _i64, _i64, _i32, _vp, _vp, _vp]),
        "lb_synth_volume": (_i32, [_vp, _vp, _vp, _vp, _i32, _i32, _i32, _f64, _i32, _vp, _vp, _vp]),
        "lb_population_sums_noalloc": (_i32, [_vp, _i32, _i32, _vp, _vp]),
        "lb_mlp_param_bytes": (_sz, [_i32]),
        "lb_mlp_bind": (_i32, [_vp, _vp, _f64]),
        "lb_mlp_train_bytes": (_sz, [_i32, _i64]),
        "lb_mlp_train_init": (_i32, [_vp, _i32, _i64, _vp, _vp]),
        "lb_mlp_features": (_i32, [_vp, _vp, _vp, _vp, _i32, _i32, _f64, _vp, _vp]),
        "lb_mlp_targets": (_i32, [_vp, _vp, _vp, _vp, _vp, _i32, _i32, _i32, _i32, _f64, _vp, _vp]),
        "lb_mlp_forward": (_i32, [_vp, _i32, _vp, _i64, _vp, _vp]),
        "lb_mlp_grad": (_i32, [_vp, _i32, _i64, _vp, _vp, _i64, _vp, _vp, _vp]),
        "lb_mlp_train_step": (_i32, [_vp, _i32, _i64, _vp, _vp, _i64, ctypes.c_float, _i64, _vp, _vp]),
        "lb_mlp_export": (_i32, [_vp, _i32, _i64, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code: int, ctx=None):
    if code != LB_OK:
        msg = load().lb_last_error(ctx)
        raise LBError(code, msg.decode() if msg else "")


def _ptr(x):
    """Device or host address of a torch tensor or numpy array (or an int)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("lbtracer needs a CUDA device; there is no CPU fallback")
    return torch


def box_desc(E, tau, periodic=(False, False, False), time_interp=LB_TIME_LINEAR, K=1, nbeads=0, rho_b=1.0,
             accel=(0.0, 0.0, 0.0), zoom=1, frame_accel=False) -> lb_box_desc:
    d = lb_box_desc()
    d.E = int(E)
    d.zoom = int(zoom)
    d.frame_accel = 1 if frame_accel else 0
    for a in range(3):
        m = LB_FACE_PERIODIC if periodic[a] else LB_FACE_VELOCITY
        d.face_mode[2 * a] = m
        d.face_mode[2 * a + 1] = m
        d.body_accel[a] = float(accel[a])
    d.time_interp = int(time_interp)
    d.K = int(K)
    d.nbeads = int(nbeads)
    d.tau = float(tau)
    d.rho_b = float(rho_b)
    return d


def chain_desc(nbeads, k_fene=30.0, R0=1.5, zeta=1.0, mass=1.0, kT=0.0, seed=0, n_md=50, pin_com=2,
               f_ext=(0.0, 0.0, 0.0), eps=1.0, sigma=1.0) -> lb_chain_desc:
    c = lb_chain_desc()
    c.nbeads, c.n_md, c.pin_com = int(nbeads), int(n_md), int(pin_com)
    c.k_fene, c.R0, c.zeta, c.mass, c.kT = float(k_fene), float(R0), float(zeta), float(mass), float(kT)
    c.eps, c.sigma = float(eps), float(sigma)
    for a in range(3):
        c.f_ext[a] = float(f_ext[a])
    c.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return c


class Tracers:
    """A context of one or more tracer boxes on one GPU.

    boxes: list of lb_box_desc; storage: LB_STORE_*; stream: torch.cuda.Stream
    (default: a new stream on the current device); ring_slots: depth of the
    boundary-sample ring (0 = 4).
    """

    def __init__(self, boxes, storage=LB_STORE_F32, stream=None, ring_slots=0):
        torch = _torch()
        lib = load()
        self.torch = torch
        self.lib = lib
        self.storage = storage
        self.descs = list(boxes)
        arr = (lb_box_desc * len(self.descs))(*self.descs)
        self._arr = arr
        nbytes = _sz()
        _check(lib.lb_plan(arr, len(self.descs), storage, int(ring_slots), ctypes.byref(nbytes)))
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.arena = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.stream.device)
        # the arena may reuse memory that work still pending on torch's current
        # stream reads; the context's own stream must come after that work
        self._after_current()
        ctx = _vp()
        _check(lib.lb_create(arr, len(self.descs), storage, int(ring_slots), self.arena.data_ptr(), nbytes.value,
                             self.stream.cuda_stream, ctypes.byref(ctx)))
        self.ctx = ctx
        self.real = torch.float64 if storage == LB_STORE_F64 else torch.float32
        self.np_real = np.float64 if storage == LB_STORE_F64 else np.float32

    def _after_current(self, *tensors):
        """Order the context stream after the work queued so far on torch's
        current stream when device memory that stream produced (or last used)
        is handed to the library: torch enqueues on its current stream, the
        library on the context's stream."""
        if tensors and not any(getattr(t, "is_cuda", False) for t in tensors):
            return
        cur = self.torch.cuda.current_stream(self.stream.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    # ---- thin wrappers (same names as the C ABI) ----
    def lb_init(self, box, u0):
        self._after_current(u0)
        _check(self.lib.lb_init(self.ctx, box, _ptr(u0)), self.ctx)

    def lb_set_boundary(self, box, j, face_u):
        self._after_current(face_u)
        _check(self.lib.lb_set_boundary(self.ctx, box, int(j), _ptr(face_u)), self.ctx)

    def chain_couple(self, box, desc: lb_chain_desc, pos0, vel0=None):
        self._after_current(pos0, vel0)
        _check(self.lib.chain_couple(self.ctx, box, ctypes.byref(desc), _ptr(pos0), _ptr(vel0)), self.ctx)

    def lb_step(self, nsteps=1):
        _check(self.lib.lb_step(self.ctx, int(nsteps)), self.ctx)

    def lb_graph_capture(self, nsteps):
        _check(self.lib.lb_graph_capture(self.ctx, int(nsteps)), self.ctx)

    def lb_graph_launch(self):
        _check(self.lib.lb_graph_launch(self.ctx), self.ctx)

    def lb_read_fields(self, box, what, dst):
        self._after_current(dst)
        _check(self.lib.lb_read_fields(self.ctx, box, what, _ptr(dst)), self.ctx)

    def lb_conservation(self, box):
        out = np.zeros(7)
        _check(self.lib.lb_conservation(self.ctx, box, out.ctypes.data), self.ctx)
        return out

    def lb_checkpoint_bytes(self):
        return int(self.lib.lb_checkpoint_bytes(self.ctx))

    def lb_save(self, dst):
        """Checkpoint of the context into dst (host numpy uint8 or device tensor of lb_checkpoint_bytes)."""
        self._after_current(dst)
        _check(self.lib.lb_save(self.ctx, _ptr(dst)), self.ctx)

    def lb_load(self, src):
        self._after_current(src)
        _check(self.lib.lb_load(self.ctx, _ptr(src)), self.ctx)

    def lb_set_frame_accel(self, box, j, a):
        """Frame-acceleration sample j (3 values, -dv/dt at t = jK) of a box created with frame_accel."""
        arr = np.ascontiguousarray(a, dtype=np.float64).reshape(3)
        _check(self.lib.lb_set_frame_accel(self.ctx, int(box), int(j), arr.ctypes.data), self.ctx)

    def lb_vorticity(self, box, lo, hi):
        """Mean |curl u| over the sites lo <= x, y, z <= hi of a box."""
        out = np.zeros(1)
        _check(self.lib.lb_vorticity(self.ctx, box, int(lo), int(hi), out.ctypes.data), self.ctx)
        return float(out[0])

    def lb_sync(self, timeout_ms=120000):
        _check(self.lib.lb_sync(self.ctx, int(timeout_ms)), self.ctx)

    def lb_status(self, box):
        st = _i32()
        _check(self.lib.lb_status(self.ctx, box, ctypes.byref(st)), self.ctx)
        return int(st.value)

    def lb_current_step(self):
        return int(self.lib.lb_current_step(self.ctx))

    def lb_set_bead_launch(self, lanes=0, beads_per_thread=1):
        _check(self.lib.lb_set_bead_launch(self.ctx, int(lanes), int(beads_per_thread)), self.ctx)

    def lb_set_chain_history(self, dev, slots):
        """Trajectory ring of the chains: dev a device float64 tensor of slots x 3 x total bead capacity
        (None with slots = 0 to stop)."""
        if dev is not None:
            self._after_current(dev)
        _check(self.lib.lb_set_chain_history(self.ctx, _ptr(dev), int(slots)), self.ctx)

    def lb_set_launch(self, kernel=LB_KERNEL_STAGED, threads=0, ctas=0, sites_per_thread=0):
        _check(self.lib.lb_set_launch(self.ctx, int(kernel), int(threads), int(ctas), int(sites_per_thread)),
               self.ctx)

    def lb_set_fluctuation(self, box, kT, seed, gamma):
        """Fluctuating collision of a box: gamma 19 relaxation factors (0..3 ignored), or None for BGK."""
        g = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.float64).reshape(19)
        _check(self.lib.lb_set_fluctuation(self.ctx, int(box), float(kT), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                           None if g is None else g.ctypes.data), self.ctx)

    def lb_test_inject(self, what, wait_limit_us=0):
        _check(self.lib.lb_test_inject(self.ctx, int(what), int(wait_limit_us)), self.ctx)

    def lb_profile(self, enable, max_launches=0):
        _check(self.lib.lb_profile(self.ctx, int(enable), int(max_launches)), self.ctx)

    def lb_profile_read(self):
        ms, n = _f64(), _i64()
        _check(self.lib.lb_profile_read(self.ctx, ctypes.byref(ms), ctypes.byref(n)), self.ctx)
        return float(ms.value), int(n.value)

    def lb_mlp_bind(self, params, u_max):
        self._after_current(params)
        _check(self.lib.lb_mlp_bind(self.ctx, _ptr(params), float(u_max)), self.ctx)

    def lb_destroy(self):
        if self.ctx:
            self.lib.lb_destroy(self.ctx)
            self.ctx = None

    # ---- conveniences ----
    def E(self, box):
        return self.descs[box].E

    def fields(self, box):
        """(rho [E,E,E], u [3,E,E,E]) as numpy arrays of the storage's real type."""
        E = self.E(box)
        rho = np.zeros((E, E, E), self.np_real)
        u = np.zeros((3, E, E, E), self.np_real)
        self.lb_read_fields(box, LB_FIELD_RHO, rho)
        self.lb_read_fields(box, LB_FIELD_U, u)
        return rho, u

    def deviations(self, box):
        E = self.E(box)
        d = np.zeros((19, E, E, E), self.np_real)
        self.lb_read_fields(box, LB_FIELD_DEV, d)
        return d

    def chain(self, box, nbeads):
        out = np.zeros((2, nbeads, 3))
        self.lb_read_fields(box, LB_FIELD_CHAIN, out)
        return out[0], out[1]

    def close(self):
        self.lb_destroy()

    def __del__(self):
        try:
            self.lb_destroy()
        except Exception:
            pass


_STORAGE_ELEM_BYTES = {LB_STORE_F64: 8, LB_STORE_F32: 4, LB_STORE_F16DEV: 2, LB_STORE_BF16DEV: 2}


def check_noalloc_args(populations, storage, E, out):
    """The C call takes no buffer sizes, so the binding checks what it can
    before any launch: populations a CUDA tensor of at least 19 E^3 elements
    whose element size matches `storage`, out a CUDA float64 tensor of at
    least 4 elements.  Raises LBError(LB_ERR_ARG) on a mismatch."""
    import torch

    def bad(msg):
        raise LBError(LB_ERR_ARG, "lb_population_sums_noalloc: " + msg)

    if int(storage) not in _STORAGE_ELEM_BYTES:
        bad("unknown storage %r" % (storage,))
    if int(E) < 1:
        bad("E must be >= 1")
    if not getattr(populations, "is_cuda", False):
        bad("populations must be a CUDA tensor")
    if populations.numel() < 19 * int(E) ** 3:
        bad("populations hold %d elements, need 19 E^3 = %d" % (populations.numel(), 19 * int(E) ** 3))
    if populations.element_size() != _STORAGE_ELEM_BYTES[int(storage)]:
        bad("element size %d does not match storage %d" % (populations.element_size(), int(storage)))
    if not getattr(out, "is_cuda", False):
        bad("out must be a CUDA tensor")
    if out.dtype != torch.float64:
        bad("out must be float64")
    if out.numel() < 4:
        bad("out must hold 4 doubles")


def lb_population_sums_noalloc(populations, storage, E, out, stream=None):
    """Mass and momentum sums of a device population buffer into the device
    tensor out (4 doubles) without any device allocation (see the C header)."""
    check_noalloc_args(populations, storage, E, out)
    torch = _torch()
    stream = stream or torch.cuda.current_stream()
    _check(load().lb_population_sums_noalloc(_ptr(populations), int(storage), int(E), _ptr(out), stream.cuda_stream))


class Upsampler:
    """Training and inference of the learned boundary upsampler on the GPU
    (thin wrapper of the lb_mlp_* calls; torch tensors hold the buffers)."""

    def __init__(self, K=16, batch_rows=16384, master=None, seed=0):
        torch = _torch()
        lib = load()
        self.torch, self.lib, self.K, self.batch = torch, lib, int(K), int(batch_rows)
        self.ws = torch.zeros(int(lib.lb_mlp_train_bytes(self.K, self.batch)), dtype=torch.uint8, device="cuda")
        self.params = torch.zeros(int(lib.lb_mlp_param_bytes(self.K)), dtype=torch.uint8, device="cuda")
        if master is None:
            raise ValueError("master parameters (float32, master layout) are required")
        m = torch.as_tensor(np.ascontiguousarray(master, np.float32)).to("cuda")
        self.stream = torch.cuda.current_stream()
        _check(lib.lb_mlp_train_init(self.ws.data_ptr(), self.K, self.batch, m.data_ptr(), self.stream.cuda_stream))
        self.t = 0
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")

    def nmaster(self):
        return 32 * 128 + 128 + 128 * 128 + 128 + 128 * 3 * self.K + 3 * self.K

    def grad(self, X, T, rows=None):
        rows = X.shape[0] if rows is None else rows
        g = self.torch.zeros(self.nmaster(), dtype=self.torch.float32, device="cuda")
        _check(self.lib.lb_mlp_grad(self.ws.data_ptr(), self.K, self.batch, X.data_ptr(), T.data_ptr(), int(rows),
                                    g.data_ptr(), self.loss.data_ptr(), self.stream.cuda_stream))
        return g, self.loss

    def step(self, X, T, lr, rows=None):
        rows = X.shape[0] if rows is None else rows
        self.t += 1
        _check(self.lib.lb_mlp_train_step(self.ws.data_ptr(), self.K, self.batch, X.data_ptr(), T.data_ptr(),
                                          int(rows), float(lr), self.t, self.loss.data_ptr(), self.stream.cuda_stream))
        return self.loss

    def export(self):
        _check(self.lib.lb_mlp_export(self.ws.data_ptr(), self.K, self.batch, self.params.data_ptr(),
                                      self.stream.cuda_stream))
        return self.params


def mlp_features(s_prev, s0, s1, s2, E, u_max, out=None):
    """bf16 features [6 E^2][32] of one face set (four [6][3][E][E] tensors)."""
    torch = _torch()
    X = out if out is not None else torch.empty((6 * E * E, 32), dtype=torch.bfloat16, device="cuda")
    code = LB_STORE_F64 if s0.dtype == torch.float64 else LB_STORE_F32
    _check(load().lb_mlp_features(s_prev.data_ptr(), s0.data_ptr(), s1.data_ptr(), s2.data_ptr(), code, int(E),
                                  float(u_max), X.data_ptr(), torch.cuda.current_stream().cuda_stream))
    return X


def mlp_targets(s_prev, s0, s1, s2, fine, E, K, first_interval, u_max, out=None):
    """f32 targets [6 E^2][3K]; fine [K+1][6][3][E][E] from t = jK."""
    torch = _torch()
    T = out if out is not None else torch.empty((6 * E * E, 3 * K), dtype=torch.float32, device="cuda")
    code = LB_STORE_F64 if s0.dtype == torch.float64 else LB_STORE_F32
    _check(load().lb_mlp_targets(s_prev.data_ptr(), s0.data_ptr(), s1.data_ptr(), s2.data_ptr(), fine.data_ptr(),
                                 code, int(E), int(K), int(first_interval), float(u_max), T.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream))
    return T


def mlp_forward(params, K, X):
    torch = _torch()
    Y = torch.empty((X.shape[0], 3 * K), dtype=torch.float32, device="cuda")
    _check(load().lb_mlp_forward(params.data_ptr(), int(K), X.data_ptr(), int(X.shape[0]), Y.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream))
    return Y


def modes_to_device(modes, device="cuda"):
    """Mode table (inputs.Modes) as four float64 device tensors."""
    torch = _torch()
    return tuple(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)
                 for a in (modes.kvec, modes.amp, modes.omega, modes.phi))


def coarse_points(E, zoom=1):
    """Points per axis of the coarse grid of a box with this zoom: point P at
    site P zoom, enough points to cover site E - 1 (E for zoom <= 1)."""
    return (E - 1 + zoom - 1) // zoom + 1 if zoom > 1 else E


def synth_faces(modes, E, K, j0, nsamp, dtype, stream=None, out=None, zoom=1):
    """Coarse face samples [nsamp][6][3][Ec][Ec] of the synthetic flow on the
    GPU (every zoom-th site; Ec = E for zoom 1)."""
    torch = _torch()
    lib = load()
    stream = stream or torch.cuda.current_stream()
    kv, am, om, ph = modes_to_device(modes)
    Ec = coarse_points(E, zoom)
    if out is None:
        out = torch.empty((nsamp, 6, 3, Ec, Ec), dtype=dtype, device="cuda")
    ws = torch.empty(int(lib.lb_synth_workspace_bytes(modes.M, E)), dtype=torch.uint8, device="cuda")
    code = LB_STORE_F64 if dtype == torch.float64 else LB_STORE_F32
    with torch.cuda.stream(stream):
        _check(lib.lb_synth_faces(kv.data_ptr(), am.data_ptr(), om.data_ptr(), ph.data_ptr(), modes.M, E, zoom, K,
                                  j0, nsamp, code, out.data_ptr(), ws.data_ptr(), stream.cuda_stream))
    stream.synchronize()
    return out


def synth_volume(modes, E, t, dtype, stream=None, zoom=1):
    """The synthetic flow at time t on the coarse grid: [3][Ec][Ec][Ec] on the
    GPU (every site for zoom 1)."""
    torch = _torch()
    lib = load()
    stream = stream or torch.cuda.current_stream()
    kv, am, om, ph = modes_to_device(modes)
    Ec = coarse_points(E, zoom)
    out = torch.empty((3, Ec, Ec, Ec), dtype=dtype, device="cuda")
    ws = torch.empty(int(lib.lb_synth_workspace_bytes(modes.M, E)), dtype=torch.uint8, device="cuda")
    code = LB_STORE_F64 if dtype == torch.float64 else LB_STORE_F32
    _check(lib.lb_synth_volume(kv.data_ptr(), am.data_ptr(), om.data_ptr(), ph.data_ptr(), modes.M, E, zoom,
                               float(t), code, out.data_ptr(), ws.data_ptr(), stream.cuda_stream))
    stream.synchronize()
    return out
