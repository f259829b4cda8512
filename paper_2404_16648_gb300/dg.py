"""Thin ctypes binding of the C ABI in ``include/dg.h`` (argument marshalling only).

Every step of the hot path runs in the CUDA kernels of ``libdg.so``; this module only converts
Python/NumPy/PyTorch arguments to the C structs and pointers.  There is no CPU fallback: if
the library is missing, importing or constructing a :class:`Mesh` raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdg.so")

DG_OK, DG_ERR_ARG, DG_ERR_CUDA, DG_ERR_OOM, DG_ERR_STATE, DG_ERR_TIMEOUT, DG_ERR_UNSUPPORTED = range(7)
DG_FP64, DG_FP32_PERT = 0, 1
DG_HOST, DG_DEVICE = 0, 1
DG_LAYOUT_PLANES, DG_LAYOUT_ELEMENTS = 0, 1
DG_CRIT_THETA, DG_CRIT_FLAGS = 0, 1
NUM_INTEGRALS = 5
STATUS_NAMES = {0: "DG_OK", 1: "DG_ERR_ARG", 2: "DG_ERR_CUDA", 3: "DG_ERR_OOM", 4: "DG_ERR_STATE",
                5: "DG_ERR_TIMEOUT", 6: "DG_ERR_UNSUPPORTED"}

# every symbol include/dg.h declares
EXPORTED = ["dg_mesh_create", "dg_mesh_destroy", "dg_num_elements", "dg_num_nodes", "dg_get_leaves",
            "dg_get_faces", "dg_set_state", "dg_get_state", "dg_set_state_async", "dg_get_state_async",
            "dg_integrals_async", "dg_get_pprime", "dg_set_vortex", "dg_set_bubble", "dg_rhs", "dg_step",
            "dg_adapt", "dg_indicator", "dg_primitives", "dg_integrals", "dg_set_time", "dg_get_time", "dg_set_option", "dg_enable_timing", "dg_stage_timing",
            "dg_forest_create_periodic", "dg_forest_create", "dg_forest_destroy", "dg_forest_size", "dg_forest_leaves",
            "dg_forest_faces", "dg_forest_regrid", "dg_integrals_noalloc", "dg_rhs_vjp",
            "dg_step_state", "dg_step_vjp", "dg_step_record", "dg_step_vjp_record", "dg_set_theta", "dg_theta_vjp", "dg_ke_grad",
            "dg_bubble_theta", "dg_forest_partition", "dg_forest_halo", "dg_batch_create", "dg_batch_destroy", "dg_batch_set_dt",
            "dg_batch_run", "dg_batch_sync", "dg_batch_autotune", "dg_batch_shape", "dg_batch_last_error",
            "dg_set_partition", "dg_get_partition", "dg_halo_pack", "dg_halo_unpack", "dg_stage_buffer",
            "dg_stage", "dg_sphere_geometry", "dg_sphere_transfer", "dg_probe_recip_sqrt", "dg_probe_fma_rate", "dg_last_error",
            "dg_version"]


class MeshDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("N", ctypes.c_int32), ("base", ctypes.c_int32 * 3),
                ("length", ctypes.c_double * 3), ("max_level", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("theta0", ctypes.c_double), ("p0", ctypes.c_double),
                ("g", ctypes.c_double), ("R", ctypes.c_double), ("cp", ctypes.c_double),
                ("nu", ctypes.c_double), ("equations", ctypes.c_int32), ("face_mode", ctypes.c_int32),
                ("wind_period", ctypes.c_double), ("periodic", ctypes.c_int32 * 3)]


class BubbleDesc(ctypes.Structure):
    _fields_ = [("center", ctypes.c_double * 3), ("radius", ctypes.c_double * 3),
                ("amp", ctypes.c_double), ("n_rff", ctypes.c_int32), ("rff_sigma", ctypes.c_double),
                ("rff_k", ctypes.POINTER(ctypes.c_double)),
                ("rff_phase", ctypes.POINTER(ctypes.c_double))]


class VortexDesc(ctypes.Structure):
    _fields_ = [("center", ctypes.c_double * 2), ("beta", ctypes.c_double),
                ("u_inf", ctypes.c_double * 2), ("t", ctypes.c_double)]


class AdaptParams(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_double), ("buffer", ctypes.c_int32),
                ("max_level", ctypes.c_int32), ("criterion", ctypes.c_int32),
                ("flags", ctypes.POINTER(ctypes.c_uint8))]


class AdaptReport(ctypes.Structure):
    _fields_ = [("elements_before", ctypes.c_int64), ("elements_after", ctypes.c_int64),
                ("refined", ctypes.c_int64), ("coarsened", ctypes.c_int64)]


class DGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def load_library(path=None):
    """Loads libdg.so (raises OSError if it was not built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError("libdg.so not built at %s; run __graft_entry__.build()" % p)
    lib = ctypes.CDLL(p)
    vp, i32, i64, sz, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
    sigs = {
        "dg_mesh_create": (i32, [ctypes.POINTER(MeshDesc), vp, ctypes.POINTER(vp)]),
        "dg_mesh_destroy": (None, [vp]),
        "dg_num_elements": (i64, [vp]),
        "dg_num_nodes": (i64, [vp]),
        "dg_get_leaves": (i32, [vp, ctypes.POINTER(ctypes.c_int32), sz]),
        "dg_get_faces": (i32, [vp, ctypes.POINTER(ctypes.c_int64), vp, sz, vp, sz, vp, sz]),
        "dg_set_state": (i32, [vp, vp, ctypes.c_int, ctypes.c_int]),
        "dg_get_state": (i32, [vp, vp, ctypes.c_int, ctypes.c_int]),
        "dg_set_state_async": (i32, [vp, vp, ctypes.c_int, vp]),
        "dg_get_state_async": (i32, [vp, vp, ctypes.c_int, vp]),
        "dg_integrals_async": (i32, [vp, vp, vp]),
        "dg_get_pprime": (i32, [vp, vp, ctypes.c_int]),
        "dg_set_bubble": (i32, [vp, ctypes.POINTER(BubbleDesc)]),
        "dg_set_vortex": (i32, [vp, ctypes.POINTER(VortexDesc)]),
        "dg_rhs": (i32, [vp, vp, vp, vp]),
        "dg_step": (i32, [vp, dbl, i32, vp]),
        "dg_adapt": (i32, [vp, ctypes.POINTER(AdaptParams), ctypes.POINTER(AdaptReport)]),
        "dg_indicator": (i32, [vp, ctypes.POINTER(ctypes.c_double), sz]),
        "dg_primitives": (i32, [vp, vp, sz, vp]),
        "dg_integrals": (i32, [vp, ctypes.POINTER(ctypes.c_double)]),
        "dg_set_option": (i32, [vp, i32, i64]),
        "dg_set_time": (i32, [vp, ctypes.c_double]),
        "dg_get_time": (ctypes.c_double, [vp]),
        "dg_enable_timing": (i32, [vp, i32]),
        "dg_stage_timing": (i32, [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), i32]),
        "dg_forest_create": (i32, [i32, ctypes.POINTER(ctypes.c_int32), i32, ctypes.POINTER(vp)]),
        "dg_forest_create_periodic": (i32, [i32, ctypes.POINTER(ctypes.c_int32), i32, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(vp)]),
        "dg_forest_destroy": (None, [vp]),
        "dg_forest_size": (i64, [vp]),
        "dg_forest_leaves": (i32, [vp, ctypes.POINTER(ctypes.c_int32), sz]),
        "dg_forest_faces": (i32, [vp, ctypes.POINTER(ctypes.c_int64), vp, sz, vp, sz, vp, sz]),
        "dg_forest_regrid": (i32, [vp, ctypes.POINTER(ctypes.c_uint8), i32, i32, vp, sz,
                                   ctypes.POINTER(ctypes.c_int64)]),
        "dg_integrals_noalloc": (i32, [ctypes.POINTER(MeshDesc), vp, i64, vp, vp, vp]),
        "dg_rhs_vjp": (i32, [vp, vp, vp, vp, vp]),
        "dg_step_state": (i32, [vp, vp, vp, dbl, i32, vp]),
        "dg_step_vjp": (i32, [vp, vp, dbl, vp, vp, vp]),
        "dg_step_record": (i32, [vp, vp, vp, vp, ctypes.c_double, vp]),
        "dg_step_vjp_record": (i32, [vp, vp, ctypes.c_double, vp, vp, vp]),
        "dg_set_theta": (i32, [vp, vp, ctypes.c_int]),
        "dg_theta_vjp": (i32, [vp, vp, vp, vp, vp]),
        "dg_ke_grad": (i32, [vp, vp, vp, vp]),
        "dg_bubble_theta": (i32, [vp, ctypes.POINTER(BubbleDesc), vp]),
        "dg_forest_partition": (i32, [vp, i32, ctypes.POINTER(ctypes.c_int64)]),
        "dg_forest_halo": (i32, [vp, i32, i32, vp, sz, ctypes.POINTER(ctypes.c_int64)]),
        "dg_batch_create": (i32, [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)]),
        "dg_batch_destroy": (None, [vp]),
        "dg_batch_set_dt": (i32, [vp, ctypes.POINTER(ctypes.c_double)]),
        "dg_batch_run": (i32, [vp, i32, i32]),
        "dg_batch_sync": (i32, [vp]),
        "dg_batch_autotune": (i32, [vp, i32, ctypes.POINTER(ctypes.c_int32)]),
        "dg_batch_shape": (i32, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "dg_batch_last_error": (ctypes.c_char_p, [vp]),
        "dg_probe_fma_rate": (i32, [i32, ctypes.POINTER(ctypes.c_double), vp]),
        "dg_probe_recip_sqrt": (i32, [i64, vp, vp, vp, vp]),
        "dg_sphere_geometry": (i32, [i32, i32, dbl, vp, i64, vp, vp, vp]),
        "dg_sphere_transfer": (i32, [i32, i32, i32, ctypes.POINTER(ctypes.c_int32), i64, vp, vp, vp, i64, vp,
                                     vp, vp]),
        "dg_set_partition": (i32, [vp, i32, i32]),
        "dg_get_partition": (i32, [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "dg_halo_pack": (i32, [vp, vp, vp, vp, vp]),
        "dg_halo_unpack": (i32, [vp, vp, vp, vp, vp]),
        "dg_stage_buffer": (i32, [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "dg_stage": (i32, [vp, i32, dbl, vp]),
        "dg_last_error": (ctypes.c_char_p, [vp]),
        "dg_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _torch():
    import torch
    return torch


def _ptr(x):
    """(address, where) of a NumPy array (host) or a torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, DG_HOST
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr(), (DG_DEVICE if x.is_cuda else DG_HOST)


def make_desc(dim, N, base, length, max_level=0, precision="fp64", theta0=300.0, p0=1.0e5, g=9.81,
              R=287.0, cp=1004.5, nu=0.0, equations="euler", face_mode="mortar", wind_period=0.0,
              periodic=(False, False, False)):
    """The dg_mesh_desc of a mesh (no device call)."""
    d = MeshDesc()
    d.dim, d.N = dim, N
    for a in range(3):
        d.base[a] = int(base[a]) if a < len(base) else 1
        d.length[a] = float(length[a]) if a < len(length) else 1.0
    d.max_level = max_level
    d.precision = DG_FP64 if precision == "fp64" else DG_FP32_PERT
    d.theta0, d.p0, d.g, d.R, d.cp, d.nu = theta0, p0, g, R, cp, nu
    if equations not in ("euler", "tracer") or face_mode not in ("mortar", "interp"):
        raise ValueError("equations must be 'euler' or 'tracer', face_mode 'mortar' or 'interp'")
    d.equations = 1 if equations == "tracer" else 0
    d.face_mode = 1 if face_mode == "interp" else 0
    d.wind_period = wind_period
    for a in range(3):
        d.periodic[a] = 1 if a < len(periodic) and periodic[a] else 0
    return d


def probe_fma_rate(precision="fp64"):
    """Measured FMA throughput of the current device in FLOP/s (dg_probe_fma_rate)."""
    lib = load_library()
    out = ctypes.c_double()
    st = lib.dg_probe_fma_rate(DG_FP64 if precision == "fp64" else DG_FP32_PERT, ctypes.byref(out), None)
    if st != DG_OK:
        raise DGError(st, "dg_probe_fma_rate failed")
    return out.value


class Mesh:
    """A forest-of-trees dGSEM mesh with its state on the GPU (one dg_mesh handle)."""

    def __init__(self, dim, N, base, length, max_level=0, precision="fp64", theta0=300.0,
                 p0=1.0e5, g=9.81, R=287.0, cp=1004.5, nu=0.0, stream=None, equations="euler",
                 face_mode="mortar", wind_period=0.0, periodic=(False, False, False)):
        self.lib = load_library()
        d = make_desc(dim, N, base, length, max_level, precision, theta0, p0, g, R, cp, nu,
                      equations, face_mode, wind_period, periodic)
        self.desc = d
        self.equations = equations
        self.dim, self.N, self.nv = dim, N, (1 if equations == "tracer" else dim + 2)
        self.np_ = (N + 1) ** dim
        self.precision = precision
        self.np_dtype = np.float64 if precision == "fp64" else np.float32
        h = ctypes.c_void_p()
        self._stream = stream
        st = self.lib.dg_mesh_create(ctypes.byref(d), self._stream_ptr(stream), ctypes.byref(h))
        if st != DG_OK:
            raise DGError(st, "dg_mesh_create failed")
        self.h = h

    # ------------------------------------------------------------------ plumbing
    def _stream_ptr(self, stream):
        if stream is None:
            return None
        return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))

    def _check(self, st):
        if st != DG_OK:
            raise DGError(st, self.lib.dg_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.dg_mesh_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ queries
    @property
    def num_elements(self):
        return int(self.lib.dg_num_elements(self.h))

    @property
    def num_nodes(self):
        return int(self.lib.dg_num_nodes(self.h))

    @property
    def num_mortars(self):
        counts = (ctypes.c_int64 * 3)()
        self._check(self.lib.dg_get_faces(self.h, counts, None, 0, None, 0, None, 0))
        return int(counts[1])

    @property
    def state_shape(self):
        return (self.nv, self.num_elements, self.np_)

    def leaves(self):
        E = self.num_elements
        out = np.zeros((E, 5), dtype=np.int32)
        self._check(self.lib.dg_get_leaves(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), out.size))
        return out

    def faces(self):
        counts = (ctypes.c_int64 * 3)()
        self._check(self.lib.dg_get_faces(self.h, counts, None, 0, None, 0, None, 0))
        c = np.zeros((counts[0], 3), np.int32)
        m = np.zeros((counts[1], 7), np.int32)
        b = np.zeros((counts[2], 3), np.int32)
        self._check(self.lib.dg_get_faces(self.h, counts, c.ctypes.data, counts[0], m.ctypes.data,
                                          counts[1], b.ctypes.data, counts[2]))
        return c, m, b

    # ------------------------------------------------------------------ state
    def _layout(self, layout):
        """(layout flag, expected shape): "planes" [nv][E][NP] (the library's), "elements"
        [E][nv][NP]."""
        if layout == "planes":
            return DG_LAYOUT_PLANES, self.state_shape
        if layout == "elements":
            nv, E, NP = self.state_shape
            return DG_LAYOUT_ELEMENTS, (E, nv, NP)
        raise ValueError("layout must be 'planes' or 'elements'")

    def set_state(self, q, layout="planes"):
        flag, shape = self._layout(layout)
        if tuple(q.shape) != shape:
            raise ValueError("state shape %s != %s" % (tuple(q.shape), shape))
        if isinstance(q, np.ndarray) and q.dtype != self.np_dtype:
            raise ValueError("state dtype must be %s" % self.np_dtype)
        p, where = _ptr(q)
        self._check(self.lib.dg_set_state(self.h, ctypes.c_void_p(p), flag, where))

    def get_state(self, out=None, layout="planes"):
        flag, shape = self._layout(layout)
        if out is None:
            out = np.empty(shape, dtype=self.np_dtype)
        if tuple(out.shape) != shape:
            raise ValueError("output shape %s != %s" % (tuple(out.shape), shape))
        p, where = _ptr(out)
        self._check(self.lib.dg_get_state(self.h, ctypes.c_void_p(p), flag, where))
        return out

    def set_state_async(self, q, stream=None):
        """Copy in on `stream` without a host wait (q: contiguous tensor; host tensors pinned)."""
        if tuple(q.shape) != self.state_shape:
            raise ValueError("state shape %s != %s" % (tuple(q.shape), self.state_shape))
        p, where = _ptr(q)
        self._check(self.lib.dg_set_state_async(self.h, ctypes.c_void_p(p), where, self._stream_ptr(stream)))

    def get_state_async(self, out, stream=None):
        """Copy out on `stream` after the mesh stream's queued work, without a host wait."""
        p, where = _ptr(out)
        self._check(self.lib.dg_get_state_async(self.h, ctypes.c_void_p(p), where, self._stream_ptr(stream)))
        return out

    def integrals_async(self, out, stream=None):
        """The integrals into `out` (6 float64: 5 integrals and a non-finite flag; a pinned host
        or a device tensor), without a host wait."""
        self._check(self.lib.dg_integrals_async(self.h, ctypes.c_void_p(out.data_ptr()), self._stream_ptr(stream)))
        return out

    def pprime(self, out=None):
        """P' plane of the current state, shape (E, (N+1)^dim), in the state precision (host
        NumPy array unless `out` is given)."""
        if out is None:
            out = np.empty((self.num_elements, self.np_), dtype=self.np_dtype)
        p, where = _ptr(out)
        self._check(self.lib.dg_get_pprime(self.h, ctypes.c_void_p(p), where))
        return out

    def set_bubble(self, center, radius, amp, rff=None):
        self._bubble(center, radius, amp, rff, None)

    def set_vortex(self, center, beta, u_inf, t=0.0):
        """Isentropic vortex of Sec. 4.1 (nondimensional mesh constants) moved to time t."""
        v = VortexDesc()
        v.center[0], v.center[1] = float(center[0]), float(center[1])
        v.beta = float(beta)
        v.u_inf[0], v.u_inf[1] = float(u_inf[0]), float(u_inf[1])
        v.t = float(t)
        self._check(self.lib.dg_set_vortex(self.h, ctypes.byref(v)))

    def bubble_theta(self, center, radius, amp, rff=None, out=None):
        """The bubble's theta' at every node as a device FP64 tensor (elements, nodes)."""
        torch = _torch()
        if out is None:
            out = torch.empty((self.num_elements, self.np_), dtype=torch.float64, device="cuda")
        self._bubble(center, radius, amp, rff, out)
        return out

    def _bubble(self, center, radius, amp, rff, theta_out):
        b = BubbleDesc()
        for a in range(3):
            b.center[a] = float(center[a]) if a < len(center) else 0.0
            b.radius[a] = float(radius[a]) if a < len(radius) else 1.0
        b.amp = amp
        keep = []
        if rff is not None:
            sigma, kvec, phase = rff
            k3 = np.zeros((len(phase), 3))
            k3[:, :kvec.shape[1]] = kvec
            k3 = np.ascontiguousarray(k3, dtype=np.float64)
            ph = np.ascontiguousarray(phase, dtype=np.float64)
            keep = [k3, ph]
            b.n_rff = len(ph)
            b.rff_sigma = sigma
            b.rff_k = k3.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            b.rff_phase = ph.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if theta_out is None:
            self._check(self.lib.dg_set_bubble(self.h, ctypes.byref(b)))
        else:
            self._check(self.lib.dg_bubble_theta(self.h, ctypes.byref(b), ctypes.c_void_p(theta_out.data_ptr())))
        del keep

    # ------------------------------------------------------------------ hot path
    def rhs(self, q, out=None, stream=None):
        """dq/dt for a device tensor q (shape state_shape) into a device tensor."""
        torch = _torch()
        if out is None:
            out = torch.empty_like(q)
        if not (q.is_cuda and out.is_cuda):
            raise ValueError("dg_rhs takes device tensors")
        self._check(self.lib.dg_rhs(self.h, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    self._stream_ptr(stream)))
        return out

    # ------------------------------------------------------------------ adjoint (FP64)
    def rhs_vjp(self, q, lam, out=None, stream=None):
        """J(q)^T lam for device tensors."""
        torch = _torch()
        if out is None:
            out = torch.empty_like(q)
        self._check(self.lib.dg_rhs_vjp(self.h, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), self._stream_ptr(stream)))
        return out

    def step_state(self, q_in, q_out, dt, nsteps=1, stream=None):
        """nsteps SSP-RK3 steps from device tensor q_in into q_out (may be the same tensor)."""
        self._check(self.lib.dg_step_state(self.h, ctypes.c_void_p(q_in.data_ptr()),
                                           ctypes.c_void_p(q_out.data_ptr()), float(dt), int(nsteps),
                                           self._stream_ptr(stream)))
        return q_out

    def step_vjp(self, q_in, dt, lam_out, lam_in=None, stream=None):
        torch = _torch()
        if lam_in is None:
            lam_in = torch.empty_like(lam_out)
        self._check(self.lib.dg_step_vjp(self.h, ctypes.c_void_p(q_in.data_ptr()), float(dt),
                                         ctypes.c_void_p(lam_out.data_ptr()), ctypes.c_void_p(lam_in.data_ptr()),
                                         self._stream_ptr(stream)))
        return lam_in

    @property
    def record_shape(self):
        """Shape of a dg_step_record buffer: 3 stage inputs x (NV + 1) planes x elements x nodes."""
        return (3, self.nv + 1, self.num_elements, (self.N + 1) ** self.dim)

    def step_record(self, q_in, q_out, record, dt, stream=None):
        self._check(self.lib.dg_step_record(self.h, ctypes.c_void_p(q_in.data_ptr()),
                                            ctypes.c_void_p(q_out.data_ptr()),
                                            ctypes.c_void_p(record.data_ptr()), float(dt),
                                            self._stream_ptr(stream)))
        return q_out

    def step_vjp_record(self, record, dt, lam_out, lam_in=None, stream=None):
        torch = _torch()
        if lam_in is None:
            lam_in = torch.empty_like(lam_out)
        self._check(self.lib.dg_step_vjp_record(self.h, ctypes.c_void_p(record.data_ptr()), float(dt),
                                                ctypes.c_void_p(lam_out.data_ptr()),
                                                ctypes.c_void_p(lam_in.data_ptr()), self._stream_ptr(stream)))
        return lam_in

    def set_theta(self, theta):
        """Initial state from a nodal theta' field [E, (N+1)^d] (numpy or device tensor)."""
        if tuple(theta.shape) != (self.num_elements, self.np_):
            raise ValueError("theta shape must be (elements, nodes per element)")
        p, where = _ptr(theta)
        self._check(self.lib.dg_set_theta(self.h, ctypes.c_void_p(p), where))

    def theta_vjp(self, theta, lam_q, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty_like(theta)
        self._check(self.lib.dg_theta_vjp(self.h, ctypes.c_void_p(theta.data_ptr()), ctypes.c_void_p(lam_q.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), self._stream_ptr(stream)))
        return out

    def ke_grad(self, q, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty_like(q)
        self._check(self.lib.dg_ke_grad(self.h, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                        self._stream_ptr(stream)))
        return out

    def step(self, dt, nsteps=1, stream=None):
        self._check(self.lib.dg_step(self.h, float(dt), int(nsteps), self._stream_ptr(stream)))

    def adapt(self, threshold=0.0, buffer=2, max_level=-1, flags=None):
        p = AdaptParams()
        p.threshold, p.buffer, p.max_level = threshold, buffer, max_level
        keep = None
        if flags is not None:
            keep = np.ascontiguousarray(flags, dtype=np.uint8)
            if keep.size != self.num_elements:
                raise ValueError("one flag per element")
            p.criterion = DG_CRIT_FLAGS
            p.flags = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        else:
            p.criterion = DG_CRIT_THETA
        r = AdaptReport()
        self._check(self.lib.dg_adapt(self.h, ctypes.byref(p), ctypes.byref(r)))
        return {"before": r.elements_before, "after": r.elements_after, "refined": r.refined,
                "coarsened": r.coarsened}

    def indicator(self):
        out = np.zeros(self.num_elements)
        self._check(self.lib.dg_indicator(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size))
        return out

    def primitives(self, out=None, stream=None):
        """FP64 device tensor [dim + 1, E, NP]: velocity components, then theta'."""
        import torch
        shape = (self.dim + 1, self.num_elements, (self.N + 1) ** self.dim)
        if out is None:
            out = torch.empty(shape, dtype=torch.float64, device="cuda")
        if out.dtype != torch.float64 or not out.is_contiguous() or out.numel() < shape[0] * shape[1] * shape[2]:
            raise ValueError("out must be a contiguous FP64 tensor of shape %s" % (shape,))
        self._check(self.lib.dg_primitives(self.h, ctypes.c_void_p(out.data_ptr()), out.numel(),
                                           self._stream_ptr(stream)))
        return out

    def integrals(self, check=True):
        out = (ctypes.c_double * NUM_INTEGRALS)()
        st = self.lib.dg_integrals(self.h, out)
        if check:
            self._check(st)
        return np.array(list(out))

    def set_time(self, t):
        self._check(self.lib.dg_set_time(self.h, float(t)))

    def get_time(self):
        return float(self.lib.dg_get_time(self.h))

    def set_stage_kernel(self, layout):
        """0: one thread per vertical node column; 1: one thread per node; 2: column layout with
        asynchronous staging of every operand in shared memory; 3: as 2 with two threads per
        column (3D, odd N); 4: one pass per axis, two threads per node line, fluxes in registers
        (3D, odd N); 5: conforming and wall face fluxes computed once per face by a face kernel,
        then a column pass and one line pass per horizontal axis.
        Default: 4 for FP32 3D meshes, 5 for FP64 Euler meshes, 2 otherwise."""
        self._check(self.lib.dg_set_option(self.h, 1, int(layout)))

    # ------------------------------------------------------------------ sharded meshes
    def set_partition(self, nparts, part):
        self._check(self.lib.dg_set_partition(self.h, int(nparts), int(part)))
        self.nparts = int(nparts)

    def partition(self):
        """(owned range, send slots per part, receive slots per part, values per slot)."""
        n = getattr(self, "nparts", 1)
        rng = (ctypes.c_int64 * 2)()
        snd = (ctypes.c_int64 * n)()
        rcv = (ctypes.c_int64 * n)()
        sv = ctypes.c_int64()
        self._check(self.lib.dg_get_partition(self.h, rng, snd, rcv, ctypes.byref(sv)))
        return (rng[0], rng[1]), list(snd), list(rcv), sv.value

    def halo_pack(self, q, pp, sendbuf, stream=None):
        self._check(self.lib.dg_halo_pack(self.h, ctypes.c_void_p(q), ctypes.c_void_p(pp) if pp else None,
                                          ctypes.c_void_p(sendbuf.data_ptr()), self._stream_ptr(stream)))

    def halo_unpack(self, recvbuf, q, pp, stream=None):
        self._check(self.lib.dg_halo_unpack(self.h, ctypes.c_void_p(recvbuf.data_ptr()), ctypes.c_void_p(q),
                                            ctypes.c_void_p(pp) if pp else None, self._stream_ptr(stream)))

    def stage_buffer(self, index):
        """Device addresses (q, P') of stage buffer `index` (0 = q^n)."""
        q, pp = ctypes.c_void_p(), ctypes.c_void_p()
        self._check(self.lib.dg_stage_buffer(self.h, int(index), ctypes.byref(q), ctypes.byref(pp)))
        return q.value, pp.value

    def stage(self, stage, dt, stream=None):
        self._check(self.lib.dg_stage(self.h, int(stage), float(dt), self._stream_ptr(stream)))

    def fail_next_adapt(self, where):
        """Host-side failure injection for the next adapt (DG_OPT_FAIL_NEXT_ADAPT): 1 fails
        before the new tree is committed, 2 after it (the mesh is then unusable)."""
        self._check(self.lib.dg_set_option(self.h, 2, int(where)))

    def enable_timing(self, on=True):
        self._check(self.lib.dg_enable_timing(self.h, 1 if on else 0))

    def stage_timing(self, reset=True):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self.lib.dg_stage_timing(self.h, ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0))
        return ms.value, n.value


class Forest:
    """Host-only handle on the library's forest (no GPU needed)."""

    def __init__(self, dim, base, max_level, periodic=(False, False, False)):
        self.lib = load_library()
        b = (ctypes.c_int32 * 3)(*[int(base[a]) if a < len(base) else 1 for a in range(3)])
        per = (ctypes.c_int32 * 3)(*[1 if a < len(periodic) and periodic[a] else 0 for a in range(3)])
        h = ctypes.c_void_p()
        st = self.lib.dg_forest_create_periodic(dim, b, max_level, per, ctypes.byref(h))
        if st != DG_OK:
            raise DGError(st, "dg_forest_create failed")
        self.h = h
        self.dim = dim

    def __len__(self):
        return int(self.lib.dg_forest_size(self.h))

    def leaves(self):
        out = np.zeros((len(self), 5), dtype=np.int32)
        st = self.lib.dg_forest_leaves(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), out.size)
        if st != DG_OK:
            raise DGError(st, "dg_forest_leaves failed")
        return out

    def faces(self):
        counts = (ctypes.c_int64 * 3)()
        self.lib.dg_forest_faces(self.h, counts, None, 0, None, 0, None, 0)
        c = np.zeros((counts[0], 3), np.int32)
        m = np.zeros((counts[1], 7), np.int32)
        b = np.zeros((counts[2], 3), np.int32)
        st = self.lib.dg_forest_faces(self.h, counts, c.ctypes.data, counts[0], m.ctypes.data,
                                      counts[1], b.ctypes.data, counts[2])
        if st != DG_OK:
            raise DGError(st, "dg_forest_faces failed")
        return c, m, b

    def regrid(self, flags, buffer, max_level=-1):
        fl = np.ascontiguousarray(flags, dtype=np.uint8)
        if fl.size != len(self):
            raise ValueError("one flag per leaf")
        cap = 9 * (len(self) << self.dim)
        tr = np.zeros(cap, dtype=np.int32)
        n = ctypes.c_int64()
        st = self.lib.dg_forest_regrid(self.h, fl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), buffer,
                                       max_level, tr.ctypes.data, cap, ctypes.byref(n))
        if st != DG_OK:
            raise DGError(st, "dg_forest_regrid failed")
        return tr[:9 * n.value].reshape(n.value, 9)

    def partition(self, nparts):
        starts = np.zeros(nparts + 1, dtype=np.int64)
        st = self.lib.dg_forest_partition(self.h, nparts, starts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        if st != DG_OK:
            raise DGError(st, "dg_forest_partition failed")
        return starts

    def halo(self, nparts, part):
        n = ctypes.c_int64()
        self.lib.dg_forest_halo(self.h, nparts, part, None, 0, ctypes.byref(n))
        rows = np.zeros((n.value, 5), dtype=np.int32)
        st = self.lib.dg_forest_halo(self.h, nparts, part, rows.ctypes.data, n.value, ctypes.byref(n))
        if st != DG_OK:
            raise DGError(st, "dg_forest_halo failed")
        return rows

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.dg_forest_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sphere_geometry(N, n, radius, leaves):
    """(W [E, (N+1)^2], area [E]) device tensors of the cubed-sphere elements whose leaf rows
    (Forest.leaves of a 6n x n forest) are given (dg_sphere_geometry)."""
    torch = _torch()
    lib = load_library()
    lv = torch.from_numpy(np.ascontiguousarray(leaves, dtype=np.int32)).cuda()
    E = lv.shape[0]
    W = torch.empty((E, (N + 1) ** 2), dtype=torch.float64, device="cuda")
    area = torch.empty(E, dtype=torch.float64, device="cuda")
    st = lib.dg_sphere_geometry(int(N), int(n), float(radius), ctypes.c_void_p(lv.data_ptr()), E,
                                ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(area.data_ptr()), None)
    if st != DG_OK:
        raise DGError(st, "dg_sphere_geometry failed")
    torch.cuda.synchronize()
    return W, area


def sphere_transfer(N, n, q_old, tmap, W_old, area_old, W_new):
    """Cubed-sphere transfer of the device fields q_old [nv, E_old, (N+1)^2] along the regrid map
    tmap (rows of Forest.regrid) into a new device tensor (dg_sphere_transfer)."""
    torch = _torch()
    lib = load_library()
    tm = np.ascontiguousarray(tmap, dtype=np.int32)
    nv, E_old = q_old.shape[0], q_old.shape[1]
    E_new = tm.shape[0]
    q_new = torch.empty((nv, E_new, q_old.shape[2]), dtype=torch.float64, device="cuda")
    st = lib.dg_sphere_transfer(int(N), int(n), int(nv), tm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), E_new,
                                ctypes.c_void_p(W_old.data_ptr()), ctypes.c_void_p(area_old.data_ptr()),
                                ctypes.c_void_p(q_old.data_ptr()), E_old, ctypes.c_void_p(W_new.data_ptr()),
                                ctypes.c_void_p(q_new.data_ptr()), None)
    if st != DG_OK:
        raise DGError(st, "dg_sphere_transfer failed")
    return q_new


class Batch:
    """Many meshes advanced together (dg_batch_*)."""

    def __init__(self, meshes, dt):
        self.lib = load_library()
        self.meshes = list(meshes)           # keep the meshes alive as long as the batch
        arr = (ctypes.c_void_p * len(self.meshes))(*[m.h.value for m in self.meshes])
        h = ctypes.c_void_p()
        st = self.lib.dg_batch_create(arr, len(self.meshes), ctypes.byref(h))
        if st != DG_OK:
            raise DGError(st, "dg_batch_create failed")
        self.h = h
        self.set_dt(dt)

    def _check(self, st):
        if st != DG_OK:
            raise DGError(st, self.lib.dg_batch_last_error(self.h).decode())

    def set_dt(self, dt):
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (len(self.meshes),)))
        self._check(self.lib.dg_batch_set_dt(self.h, d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def run(self, nsteps, graph=True, sync=True):
        self._check(self.lib.dg_batch_run(self.h, int(nsteps), 1 if graph else 0))
        if sync:
            self.sync()

    def sync(self):
        self._check(self.lib.dg_batch_sync(self.h))

    def autotune(self, reps=5):
        out = np.zeros(len(self.meshes), dtype=np.int32)
        self._check(self.lib.dg_batch_autotune(self.h, int(reps), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return out

    def shape(self):
        """The persistent launch's shapes (dg_batch_shape) as a dict."""
        out = (ctypes.c_int64 * 5)()
        self._check(self.lib.dg_batch_shape(self.h, out))
        return {"ctas_per_sm_budget": out[0], "tiles_per_item": out[1], "grid": out[2],
                "items_per_stage": out[3], "smem_bytes": out[4]}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.dg_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adapt_initial(mesh, bubble, threshold, buffer):
    """Adapts mesh.max_level times on the analytic bubble, re-evaluated after each pass."""
    for _ in range(mesh.desc.max_level):
        mesh.set_bubble(**bubble)
        mesh.adapt(threshold=threshold, buffer=buffer)
    mesh.set_bubble(**bubble)
