"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the simulation runs in the sm_103a library
``_lib/liblbm_gb300.so``; this module only converts arguments.  PyTorch is
used for the device workspace and the CUDA stream.  There is no fallback: if
the library is missing or cannot be loaded, every call raises.

The functions carry the names of the C entry points (``lbm_init``,
``lbm_step``, ``lbm_get_fields``, ...).  ``Simulation`` bundles one handle with
its workspace tensor.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# LBM_LIBRARY selects another build of the same library (the bounds-checked
# one of the tests); it is never a fallback: a missing library raises.
LIB_PATH = os.environ.get("LBM_LIBRARY") or os.path.join(_PKG, "_lib", "liblbm_gb300.so")

LBM_OK, LBM_EINVAL, LBM_ENOSPC, LBM_ENUMERIC = 0, -1, -2, -3
LBM_EBOUNDS = -8
LBM_EDOMAIN, LBM_EOVERFLOW, LBM_ETIMEOUT, LBM_ECUDA = -4, -5, -6, -7
LBM_BC_PERIODIC_X, LBM_BC_PERIODIC_Y = 1, 2
LBM_STORE_FP32, LBM_STORE_BF16, LBM_STORE_FP16 = 0, 1, 2
LBM_FLAG_FIXED_PARTICLES, LBM_FLAG_NO_GRAPH, LBM_FLAG_OVERLAP, LBM_FLAG_DIRECT_LINKS = 1, 2, 4, 8
LBM_FLAG_ALL_PAIRS = 16
LBM_FLAG_SC_UNSTAGED, LBM_FLAG_TEST_WAIT_TIMEOUT = 32, 64

PARTICLE_DTYPE = np.dtype([(n, "f8") for n in
                           ("x", "y", "ux", "uy", "theta", "omega", "r", "rho", "T", "b")])


class LbmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (where, lbm_strerror(code), code))


class lbm_domain(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("bc", C.c_uint32), ("reserved", C.c_int32),
                ("T_wall", C.c_double * 4)]


class lbm_params(C.Structure):
    _fields_ = [("nu", C.c_double), ("alpha", C.c_double), ("g", C.c_double), ("beta", C.c_double),
                ("T0", C.c_double), ("rho_f", C.c_double), ("T_init", C.c_double),
                ("s_e", C.c_double), ("s_eps", C.c_double), ("s_q", C.c_double),
                ("q_e", C.c_double), ("q_nu", C.c_double), ("eps_w", C.c_double),
                ("s_rep", C.c_double), ("body_fx", C.c_double), ("body_fy", C.c_double),
                ("storage", C.c_int32), ("flags", C.c_uint32)]


_lib = None

# (name, restype, argtypes) of every exported entry point
_P = C.c_void_p
_SIGS = [
    ("lbm_query_footprint", C.c_int, [_P, _P, C.c_int32, _P, C.POINTER(C.c_size_t)]),
    ("lbm_init", C.c_int, [C.POINTER(_P), _P, _P, C.c_int32, _P, _P, C.c_size_t, _P]),
    ("lbm_step", C.c_int, [_P, C.c_int32]),
    ("lbm_sync", C.c_int, [_P]),
    ("lbm_get_fields", C.c_int, [_P, _P, _P, _P, _P, C.c_int32]),
    ("lbm_get_particles", C.c_int, [_P, _P, C.c_int32]),
    ("lbm_get_particles_async", C.c_int, [_P, _P, C.c_int32]),
    ("lbm_get_forces", C.c_int, [_P, _P, C.c_int32]),
    ("lbm_destroy", C.c_int, [_P]),
    ("lbm_strerror", C.c_char_p, [C.c_int]),
    ("lbm_get_owner", C.c_int, [_P, _P]),
    ("lbm_get_slots", C.c_int, [_P, _P, _P, C.c_int64, C.POINTER(C.c_int64)]),
    ("lbm_state_bytes", C.c_int, [_P, C.POINTER(C.c_size_t)]),
    ("lbm_get_state", C.c_int, [_P, _P, C.c_size_t]),
    ("lbm_set_state", C.c_int, [_P, _P, C.c_size_t]),
    ("lbm_set_distributions", C.c_int, [_P, _P, _P]),
    ("lbm_get_counters", C.c_int, [_P, _P]),
    ("lbm_kernel_timing", C.c_int, [_P, C.c_int32]),
    ("lbm_kernel_times", C.c_int, [_P, _P, _P, C.c_int32]),
    ("lbm_kernel_count", C.c_int32, []),
    ("lbm_kernel_name", C.c_char_p, [C.c_int32]),
    ("lbm_launch_count", C.c_int64, [_P]),
    ("lbm_binary_version", C.c_int, [C.POINTER(C.c_int32)]),
    ("lbm_link_forces_noalloc", C.c_int, [_P, C.c_int64, C.c_int32, _P, C.c_int32, C.c_int32, _P,
                                          C.c_int32, C.c_double, _P, _P]),
    ("lbm_batch_footprint", C.c_int, [_P, C.c_int32, C.POINTER(C.c_size_t)]),
    ("lbm_batch_create", C.c_int, [C.POINTER(_P), _P, C.c_int32, _P, C.c_size_t, _P]),
    ("lbm_batch_autotune", C.c_int, [_P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    ("lbm_batch_step", C.c_int, [_P, C.c_int32]),
    ("lbm_batch_sync", C.c_int, [_P, C.POINTER(C.c_int32)]),
    ("lbm_batch_launch_count", C.c_int64, [_P]),
    ("lbm_batch_destroy", C.c_int, [_P]),
    ("lbm_server_create", C.c_int, [C.POINTER(_P), _P, C.c_size_t, C.c_int32, _P]),
    ("lbm_server_submit", C.c_int, [_P, _P, _P, C.c_int32, _P, C.c_int64, C.POINTER(C.c_int64)]),
    ("lbm_server_tick", C.c_int, [_P, C.c_int32, _P]),
    ("lbm_server_status", C.c_int, [_P, C.c_int64, C.POINTER(C.c_int32)]),
    ("lbm_server_result", C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, C.c_int32]),
    ("lbm_server_destroy", C.c_int, [_P]),
]


def library():
    """Load the CUDA library (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("the sm_103a library %s is not built; run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return [s[0] for s in _SIGS]


def _check(rc: int, where: str):
    if rc != LBM_OK:
        raise LbmError(rc, where)


def lbm_strerror(code: int) -> str:
    return library().lbm_strerror(int(code)).decode()


def make_domain(nx, ny, T_wall=(0.0, 0.0, 0.0, 0.0), periodic_x=0, periodic_y=0, **_):
    d = lbm_domain()
    d.nx, d.ny = int(nx), int(ny)
    d.bc = (LBM_BC_PERIODIC_X if periodic_x else 0) | (LBM_BC_PERIODIC_Y if periodic_y else 0)
    d.reserved = 0
    for i in range(4):
        d.T_wall[i] = float(T_wall[i])
    return d


def make_params(nu, alpha, g=0.0, beta=1.0, T0=0.0, rho_f=1.0, T_init=0.0, s_e=0.0, s_eps=0.0,
                s_q=0.0, q_e=0.0, q_nu=0.0, eps_w=1e-3, s_rep=3.0, body_fx=0.0, body_fy=0.0,
                fixed_particles=0, storage=LBM_STORE_FP32, flags=0, **_):
    p = lbm_params()
    for k, v in dict(nu=nu, alpha=alpha, g=g, beta=beta, T0=T0, rho_f=rho_f, T_init=T_init,
                     s_e=s_e, s_eps=s_eps, s_q=s_q, q_e=q_e, q_nu=q_nu, eps_w=eps_w, s_rep=s_rep,
                     body_fx=body_fx, body_fy=body_fy).items():
        setattr(p, k, float(v))
    p.storage = int(storage)
    p.flags = int(flags) | (LBM_FLAG_FIXED_PARTICLES if fixed_particles else 0)
    return p


def pack_particles(parts) -> np.ndarray:
    out = np.zeros(0 if parts is None else len(parts), PARTICLE_DTYPE)
    if parts is not None and len(parts):
        have = parts.dtype.names or ()
        for n in PARTICLE_DTYPE.names:
            if n in have:  # "b" may be absent: disks
                out[n] = np.asarray(parts[n], dtype=np.float64)
    return np.ascontiguousarray(out)


def lbm_query_footprint(domain: lbm_domain, parts: np.ndarray, params: lbm_params) -> int:
    b = C.c_size_t(0)
    _check(library().lbm_query_footprint(C.byref(domain), parts.ctypes.data if len(parts) else None,
                                         len(parts), C.byref(params), C.byref(b)),
           "lbm_query_footprint")
    return b.value


def lbm_init(domain, parts, params, workspace_ptr: int, ws_bytes: int, stream_ptr: int):
    h = C.c_void_p()
    _check(library().lbm_init(C.byref(h), C.byref(domain),
                              parts.ctypes.data if len(parts) else None, len(parts),
                              C.byref(params), C.c_void_p(workspace_ptr), ws_bytes,
                              C.c_void_p(stream_ptr)), "lbm_init")
    return h


def lbm_step(h, n: int = 1):
    _check(library().lbm_step(h, int(n)), "lbm_step")


def lbm_sync(h):
    _check(library().lbm_sync(h), "lbm_sync")


def lbm_destroy(h):
    _check(library().lbm_destroy(h), "lbm_destroy")


def lbm_get_fields(h, drho_ptr, ux_ptr, uy_ptr, T_ptr, on_device: int):
    _check(library().lbm_get_fields(h, drho_ptr, ux_ptr, uy_ptr, T_ptr, int(on_device)),
           "lbm_get_fields")


def lbm_get_particles(h, out: np.ndarray):
    _check(library().lbm_get_particles(h, out.ctypes.data if len(out) else None, len(out)),
           "lbm_get_particles")


def lbm_get_particles_async(h, out: np.ndarray):
    """Enqueue the copy of the particle states into out (page-locked for
    overlap); valid after lbm_sync."""
    _check(library().lbm_get_particles_async(h, out.ctypes.data if len(out) else None, len(out)),
           "lbm_get_particles_async")


def lbm_get_forces(h, out: np.ndarray, n: int):
    _check(library().lbm_get_forces(h, out.ctypes.data if n else None, n), "lbm_get_forces")


class Simulation:
    """One simulation: a handle plus the torch-owned device workspace."""

    def __init__(self, domain: dict, particles, params: dict, stream=None, storage=LBM_STORE_FP32,
                 flags=0, device="cuda"):
        import torch
        library()
        self.nx, self.ny = int(domain["nx"]), int(domain["ny"])
        self._domain = make_domain(**domain)
        self._params = make_params(**dict(params, storage=storage, flags=flags))
        self._parts = pack_particles(particles)
        self.np = len(self._parts)
        self.ws_bytes = lbm_query_footprint(self._domain, self._parts, self._params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        self.h = lbm_init(self._domain, self._parts, self._params, self.workspace.data_ptr(),
                          self.ws_bytes, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        lbm_step(self.h, n)

    def sync(self):
        lbm_sync(self.h)

    def fields(self):
        """drho = rho - 1, ux, uy, T as float32 numpy arrays [ny][nx] (NaN at
        solid nodes)."""
        out = [np.empty((self.ny, self.nx), np.float32) for _ in range(4)]
        lbm_get_fields(self.h, *[o.ctypes.data for o in out], 0)
        return tuple(out)

    def fields_device(self):
        import torch
        out = [torch.empty((self.ny, self.nx), dtype=torch.float32, device=self.workspace.device)
               for _ in range(4)]
        lbm_get_fields(self.h, *[o.data_ptr() for o in out], 1)
        return tuple(out)

    def particles(self, out=None) -> np.ndarray:
        if out is None:
            out = np.zeros(self.np, PARTICLE_DTYPE)
        lbm_get_particles(self.h, out)
        return out

    def forces(self) -> np.ndarray:
        out = np.zeros((self.np, 3))
        lbm_get_forces(self.h, out, self.np)
        return out

    def owner(self) -> np.ndarray:
        out = np.empty((self.ny, self.nx), np.int32)
        _check(library().lbm_get_owner(self.h, out.ctypes.data), "lbm_get_owner")
        return out

    def slots(self):
        cnt = C.c_int64(0)
        _check(library().lbm_get_slots(self.h, None, None, 0, C.byref(cnt)), "lbm_get_slots")
        node = np.empty(cnt.value, np.int32)
        q = np.empty(cnt.value, np.float32)
        _check(library().lbm_get_slots(self.h, node.ctypes.data, q.ctypes.data, cnt.value,
                                       C.byref(cnt)), "lbm_get_slots")
        return node, q

    def get_state(self) -> bytes:
        b = C.c_size_t(0)
        _check(library().lbm_state_bytes(self.h, C.byref(b)), "lbm_state_bytes")
        buf = np.empty(b.value, np.uint8)
        _check(library().lbm_get_state(self.h, buf.ctypes.data, b.value), "lbm_get_state")
        return buf

    def set_state(self, buf: np.ndarray):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(library().lbm_set_state(self.h, buf.ctypes.data, buf.size), "lbm_set_state")

    def set_distributions(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx) and g.shape == (5, self.ny, self.nx)
        _check(library().lbm_set_distributions(self.h, f.ctypes.data, g.ctypes.data),
               "lbm_set_distributions")

    def counters(self) -> np.ndarray:
        out = np.zeros(8, np.int64)
        _check(library().lbm_get_counters(self.h, out.ctypes.data), "lbm_get_counters")
        return out

    def kernel_timing(self, enable: bool):
        _check(library().lbm_kernel_timing(self.h, int(bool(enable))), "lbm_kernel_timing")

    def kernel_times(self) -> dict:
        lib = library()
        nk = lib.lbm_kernel_count()
        ms = np.zeros(nk)
        n = np.zeros(nk, np.int64)
        _check(lib.lbm_kernel_times(self.h, ms.ctypes.data, n.ctypes.data, nk), "lbm_kernel_times")
        return {lib.lbm_kernel_name(k).decode(): (float(ms[k]), int(n[k])) for k in range(nk)}

    def launch_count(self) -> int:
        return int(library().lbm_launch_count(self.h))


def lbm_binary_version() -> int:
    """GPU architecture of the loaded device code (103 for sm_103a)."""
    v = C.c_int32(0)
    _check(library().lbm_binary_version(C.byref(v)), "lbm_binary_version")
    return int(v.value)


def lbm_link_forces_noalloc(dist_ptr, plane_stride, pitch, owner_ptr, nx, ny, particles_ptr, n,
                            r_max, forces_ptr, stream_ptr):
    """Allocation-free link forces (see include/lbm.h); device pointers in."""
    _check(library().lbm_link_forces_noalloc(dist_ptr, plane_stride, pitch, owner_ptr, nx, ny,
                                             particles_ptr, n, r_max, forces_ptr, stream_ptr),
           "lbm_link_forces_noalloc")


class Batch:
    """Independent simulations stepped together: one launch per step kernel
    over all of them (lbm_batch_* in include/lbm.h).  The simulations stay
    usable on their own after sync()."""

    def __init__(self, sims, stream=None):
        import torch
        lib = library()
        self.sims = list(sims)
        n = len(self.sims)
        arr = (_P * n)(*[s.h for s in self.sims])
        self._arr = arr
        b = C.c_size_t()
        _check(lib.lbm_batch_footprint(arr, n, C.byref(b)), "lbm_batch_footprint")
        dev = self.sims[0].workspace.device
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.workspace = torch.empty(max(int(b.value), 1), dtype=torch.uint8, device=dev)
        h = _P()
        _check(lib.lbm_batch_create(C.byref(h), arr, n, self.workspace.data_ptr(), int(b.value),
                                    self.stream.cuda_stream), "lbm_batch_create")
        self.h = h

    @property
    def nodes(self) -> int:
        return sum(s.nx * s.ny for s in self.sims)

    def autotune(self, reps: int = 3) -> int:
        """Pick the stream-collide tile shape; returns its index (the mean
        time per stream-collide launch of that shape is in self.tuned_ms)."""
        c = C.c_int32()
        ms = C.c_double()
        _check(library().lbm_batch_autotune(self.h, int(reps), C.byref(c), C.byref(ms)), "lbm_batch_autotune")
        self.tuned_ms = float(ms.value)
        return int(c.value)

    def step(self, n: int = 1):
        _check(library().lbm_batch_step(self.h, int(n)), "lbm_batch_step")

    def sync(self):
        w = C.c_int32()
        rc = library().lbm_batch_sync(self.h, C.byref(w))
        _check(rc, "lbm_batch_sync (instance %d)" % w.value)

    def launch_count(self) -> int:
        return int(library().lbm_batch_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            library().lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class lbm_server_stats(C.Structure):
    _fields_ = [("active", C.c_int32), ("queued", C.c_int32), ("admitted", C.c_int32),
                ("retired", C.c_int32), ("steps", C.c_int32), ("reserved", C.c_int32),
                ("ms", C.c_double), ("updates", C.c_int64)]


SERVER_QUEUED, SERVER_ACTIVE, SERVER_DONE, SERVER_FAILED = 0, 1, 2, 3


class Server:
    """Request loop over one device memory pool (lbm_server_* in
    include/lbm.h): submit simulations with a step budget, tick to admit,
    advance and retire them, fetch the results of finished ones."""

    def __init__(self, pool_bytes: int, max_active: int = 32, stream=None, device="cuda"):
        import torch
        lib = library()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=device)
        h = _P()
        _check(lib.lbm_server_create(C.byref(h), self.pool.data_ptr(), int(pool_bytes), int(max_active),
                                     self.stream.cuda_stream), "lbm_server_create")
        self.h = h
        self._shape = {}

    def submit(self, domain: dict, particles, params: dict, steps: int, storage=LBM_STORE_FP32,
               flags=0) -> int:
        d = make_domain(**domain)
        prm = make_params(**dict(params, storage=storage, flags=flags))
        parts = pack_particles(particles)
        rid = C.c_int64()
        _check(library().lbm_server_submit(self.h, C.byref(d), parts.ctypes.data if len(parts) else None,
                                           len(parts), C.byref(prm), int(steps), C.byref(rid)),
               "lbm_server_submit")
        self._shape[rid.value] = (int(domain["ny"]), int(domain["nx"]), len(parts))
        return int(rid.value)

    def tick(self, max_steps: int) -> dict:
        st = lbm_server_stats()
        _check(library().lbm_server_tick(self.h, int(max_steps), C.byref(st)), "lbm_server_tick")
        return {k: getattr(st, k) for k, _ in st._fields_ if k != "reserved"}

    def status(self, rid: int):
        err = C.c_int32()
        state = library().lbm_server_status(self.h, int(rid), C.byref(err))
        return int(state), int(err.value)

    def result(self, rid: int):
        """(rho - 1, ux, uy, T) float32 [ny][nx] and the particles of a done
        request (which the server then forgets)."""
        ny, nx, n = self._shape[rid]
        f = [np.empty((ny, nx), np.float32) for _ in range(4)]
        parts = np.zeros(n, PARTICLE_DTYPE)
        _check(library().lbm_server_result(self.h, int(rid), *[a.ctypes.data for a in f],
                                           parts.ctypes.data if n else None, n), "lbm_server_result")
        del self._shape[rid]
        return tuple(f), parts

    def close(self):
        if getattr(self, "h", None):
            library().lbm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
