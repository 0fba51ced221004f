"""ctypes binding of the FP64 C oracle (lbm_oracle.c).

TEST INFRASTRUCTURE ONLY.  ``build()`` compiles ``lbm_oracle.c`` with gcc into
``oracle/_build/liblbm_oracle.so`` (no FMA contraction, OpenMP over the
per-node loops, which does not change any result).  ``Oracle`` wraps one
simulation; the module-level functions wrap the pure geometry routines.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_HDR = os.path.join(_HERE, "lbm_oracle.h")

ORC_PARTICLE_DTYPE = np.dtype(
    [("x", "f8"), ("y", "f8"), ("ux", "f8"), ("uy", "f8"), ("theta", "f8"),
     ("omega", "f8"), ("r", "f8"), ("rho", "f8"), ("T", "f8"), ("b", "f8")])


class _Domain(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("periodic_x", C.c_int32),
                ("periodic_y", C.c_int32), ("T_wall", C.c_double * 4)]


class _Params(C.Structure):
    _fields_ = [("nu", C.c_double), ("alpha", C.c_double), ("g", C.c_double),
                ("beta", C.c_double), ("T0", C.c_double), ("rho_f", C.c_double),
                ("T_init", C.c_double), ("s_e", C.c_double), ("s_eps", C.c_double),
                ("s_q", C.c_double), ("q_e", C.c_double), ("q_nu", C.c_double),
                ("eps_w", C.c_double), ("s_rep", C.c_double), ("body_fx", C.c_double),
                ("body_fy", C.c_double), ("fixed_particles", C.c_int32),
                ("reserved", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    fresh = (os.path.exists(_LIB_PATH)
             and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if fresh and not force:
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB_PATH)
    P = C.c_void_p
    d = C.POINTER(C.c_double)
    i32 = C.POINTER(C.c_int32)
    lib.orc_create.restype = P
    lib.orc_create.argtypes = [C.POINTER(_Domain), P, C.c_int32, C.POINTER(_Params)]
    lib.orc_destroy.argtypes = [P]
    lib.orc_step.argtypes = [P, C.c_int32]
    lib.orc_step.restype = C.c_int
    lib.orc_get_fields.argtypes = [P, d, d, d, d]
    lib.orc_get_particles.argtypes = [P, P]
    lib.orc_get_forces.argtypes = [P, d]
    lib.orc_get_owner.argtypes = [P, i32]
    lib.orc_get_state.argtypes = [P, d, d]
    lib.orc_set_state.argtypes = [P, d, d]
    lib.orc_get_counters.argtypes = [P, C.POINTER(C.c_int64)]
    lib.orc_raster.argtypes = [C.c_int32, C.c_int32, P, C.c_int32, i32]
    lib.orc_zone_size.argtypes = [C.c_double]
    lib.orc_zone_size.restype = C.c_int32
    lib.orc_slot_capacity.argtypes = [C.c_double]
    lib.orc_slot_capacity.restype = C.c_int32
    lib.orc_build_slots.argtypes = [C.c_int32, C.c_int32, i32, P, C.c_int32, i32,
                                    C.POINTER(C.c_float)]
    lib.orc_build_slots.restype = C.c_int32
    lib.orc_links_bruteforce.argtypes = [C.c_int32, C.c_int32, i32, P, C.c_int32, C.c_int64,
                                         i32, i32, i32, d]
    lib.orc_links_bruteforce.restype = C.c_int64
    lib.orc_link_q.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double,
                               C.c_double]
    lib.orc_link_q.restype = C.c_double
    lib.orc_moment_matrices.argtypes = [d, d, d, d]
    lib.orc_collide_f.argtypes = [d, C.c_double, C.c_double, C.POINTER(_Params), d]
    lib.orc_collide_g.argtypes = [d, C.c_double, C.c_double, C.POINTER(_Params), d]
    lib.orc_feq.argtypes = [C.c_double, C.c_double, C.c_double, d]
    lib.orc_geq.argtypes = [C.c_double, C.c_double, C.c_double, d]
    lib.orc_bouzidi.argtypes = [C.c_double, C.c_int32] + [C.c_double] * 5 + \
        [C.c_int32, C.c_int32, C.c_double, i32]
    lib.orc_bouzidi.restype = C.c_double
    lib.orc_thermal_bb.argtypes = [C.c_double] + [C.c_double] * 3 + [C.c_int32, C.c_double, i32]
    lib.orc_thermal_bb.restype = C.c_double
    lib.orc_repulsion.argtypes = [C.c_double] * 4
    lib.orc_repulsion.restype = C.c_double
    lib.orc_cos_sin.argtypes = [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.orc_cos_sin.restype = None
    lib.orc_in_particle.argtypes = [C.c_int32, C.c_int32, P]
    lib.orc_in_particle.restype = C.c_int32
    lib.orc_link_q_particle.argtypes = [C.c_int32, C.c_int32, C.c_int32, P]
    lib.orc_link_q_particle.restype = C.c_double
    lib.orc_support.argtypes = [P, C.c_double, C.c_double]
    lib.orc_support.restype = C.c_double
    lib.orc_integrate.argtypes = [P, C.c_double, C.c_double, C.c_double, P]
    lib.orc_refill_direction.argtypes = [C.c_double, C.c_double]
    lib.orc_refill_direction.restype = C.c_int32
    lib.orc_refill_node.argtypes = [d, d, d, C.c_int32, C.c_double, C.c_double, C.c_double,
                                    d, d, d]
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _particles(p) -> np.ndarray:
    """Any record array / dict list with the particle fields -> packed array."""
    if p is None:
        return np.zeros(0, ORC_PARTICLE_DTYPE)
    out = np.zeros(len(p), ORC_PARTICLE_DTYPE)
    for name in ORC_PARTICLE_DTYPE.names:
        if isinstance(p, list):
            if name == "b" and any(name not in q for q in p):
                continue  # disks: b = 0
            out[name] = np.asarray([q[name] for q in p], dtype=np.float64)
        else:
            if name == "b" and name not in (p.dtype.names or ()):
                continue
            out[name] = np.asarray(p[name], dtype=np.float64)
    return out


def make_params(**kw) -> _Params:
    prm = _Params()
    defaults = dict(nu=0.1, alpha=0.1, g=0.0, beta=1.0, T0=0.0, rho_f=1.0, T_init=0.0,
                    s_e=0.0, s_eps=0.0, s_q=0.0, q_e=0.0, q_nu=0.0, eps_w=1e-3, s_rep=3.0,
                    body_fx=0.0, body_fy=0.0, fixed_particles=0)
    defaults.update(kw)
    for k, v in defaults.items():
        setattr(prm, k, v)
    return prm


def make_domain(nx, ny, periodic_x=0, periodic_y=0, T_wall=(0.0, 0.0, 0.0, 0.0)) -> _Domain:
    d = _Domain()
    d.nx, d.ny, d.periodic_x, d.periodic_y = nx, ny, int(periodic_x), int(periodic_y)
    for i in range(4):
        d.T_wall[i] = T_wall[i]
    return d


class Oracle:
    """One FP64 oracle simulation; same inputs as the C-ABI's lbm_init."""

    def __init__(self, domain: dict, particles, params: dict):
        self.lib = load()
        self.nx, self.ny = int(domain["nx"]), int(domain["ny"])
        self._d = make_domain(**domain)
        self._p = make_params(**params)
        self._parts = _particles(particles)
        self.np = len(self._parts)
        self.h = self.lib.orc_create(C.byref(self._d), self._parts.ctypes.data, self.np,
                                     C.byref(self._p))

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def step(self, n: int = 1) -> int:
        return self.lib.orc_step(self.h, int(n))

    def fields(self):
        shp = (self.ny, self.nx)
        rho, ux, uy, T = (np.empty(shp) for _ in range(4))
        self.lib.orc_get_fields(self.h, _dptr(rho), _dptr(ux), _dptr(uy), _dptr(T))
        return rho, ux, uy, T

    def particles(self) -> np.ndarray:
        out = np.zeros(self.np, ORC_PARTICLE_DTYPE)
        if self.np:
            self.lib.orc_get_particles(self.h, out.ctypes.data)
        return out

    def forces(self) -> np.ndarray:
        out = np.zeros((self.np, 3))
        if self.np:
            self.lib.orc_get_forces(self.h, _dptr(out))
        return out

    def owner(self) -> np.ndarray:
        out = np.empty((self.ny, self.nx), np.int32)
        self.lib.orc_get_owner(self.h, _iptr(out))
        return out

    def state(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((5, self.ny, self.nx))
        self.lib.orc_get_state(self.h, _dptr(f), _dptr(g))
        return f, g

    def set_state(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(5, self.ny, self.nx)
        self.lib.orc_set_state(self.h, _dptr(f), _dptr(g))

    def counters(self) -> np.ndarray:
        out = np.zeros(8, np.int64)
        self.lib.orc_get_counters(self.h, out.ctypes.data_as(C.POINTER(C.c_int64)))
        return out


# --- pure geometry --------------------------------------------------------------------------
def raster(nx, ny, particles) -> np.ndarray:
    lib = load()
    p = _particles(particles)
    out = np.empty((ny, nx), np.int32)
    lib.orc_raster(nx, ny, p.ctypes.data, len(p), _iptr(out))
    return out


def zone_size(r: float) -> int:
    return load().orc_zone_size(float(r))


def slot_capacity(r: float) -> int:
    return load().orc_slot_capacity(float(r))


def build_slots(nx, ny, owner, particles):
    lib = load()
    p = _particles(particles)
    owner = np.ascontiguousarray(owner, dtype=np.int32)
    total = sum(slot_capacity(r) for r in p["r"])
    node = np.empty(total, np.int32)
    q = np.empty(total, np.float32)
    over = lib.orc_build_slots(nx, ny, _iptr(owner), p.ctypes.data, len(p), _iptr(node),
                               q.ctypes.data_as(C.POINTER(C.c_float)))
    return node, q, over


def links_bruteforce(nx, ny, owner, particles):
    lib = load()
    p = _particles(particles)
    owner = np.ascontiguousarray(owner, dtype=np.int32)
    cap = 8 * nx * ny
    while True:
        node = np.empty(cap, np.int32)
        d = np.empty(cap, np.int32)
        pid = np.empty(cap, np.int32)
        q = np.empty(cap)
        n = lib.orc_links_bruteforce(nx, ny, _iptr(owner), p.ctypes.data, len(p), cap,
                                     _iptr(node), _iptr(d), _iptr(pid), _dptr(q))
        if n <= cap:
            return node[:n], d[:n], pid[:n], q[:n]
        cap = n


def link_q(i, j, k, x, y, r) -> float:
    return load().orc_link_q(int(i), int(j), int(k), float(x), float(y), float(r))


def moment_matrices():
    M, Mi = np.empty(81), np.empty(81)
    N, Ni = np.empty(25), np.empty(25)
    load().orc_moment_matrices(_dptr(M), _dptr(Mi), _dptr(N), _dptr(Ni))
    return M.reshape(9, 9), Mi.reshape(9, 9), N.reshape(5, 5), Ni.reshape(5, 5)


def collide_f(f, Fx, Fy, **params):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty(9)
    prm = make_params(**params)
    load().orc_collide_f(_dptr(f), float(Fx), float(Fy), C.byref(prm), _dptr(out))
    return out


def collide_g(g, ux, uy, **params):
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.empty(5)
    prm = make_params(**params)
    load().orc_collide_g(_dptr(g), float(ux), float(uy), C.byref(prm), _dptr(out))
    return out


def feq(rho, ux, uy):
    out = np.empty(9)
    load().orc_feq(rho, ux, uy, _dptr(out))
    return out


def geq(T, ux, uy):
    out = np.empty(5)
    load().orc_geq(T, ux, uy, _dptr(out))
    return out


def bouzidi(q, k, fk0, fk1, fk2, fb0, fb1, have1, have2, eu):
    lvl = C.c_int32(0)
    v = load().orc_bouzidi(q, k, fk0, fk1, fk2, fb0, fb1, int(have1), int(have2), eu,
                           C.byref(lvl))
    return v, lvl.value


def thermal_bb(q, gk0, gk1, gb0, have1, Tw):
    lvl = C.c_int32(0)
    v = load().orc_thermal_bb(q, gk0, gk1, gb0, int(have1), Tw, C.byref(lvl))
    return v, lvl.value


def repulsion(gap, s, eps, Cf):
    return load().orc_repulsion(gap, s, eps, Cf)


def cos_sin(theta):
    c, s = C.c_double(), C.c_double()
    load().orc_cos_sin(float(theta), C.byref(c), C.byref(s))
    return c.value, s.value


def in_particle(i, j, particle) -> bool:
    p = _particles(particle if not isinstance(particle, dict) else [particle])
    return bool(load().orc_in_particle(int(i), int(j), p.ctypes.data))


def link_q_particle(i, j, k, particle) -> float:
    p = _particles(particle if not isinstance(particle, dict) else [particle])
    return load().orc_link_q_particle(int(i), int(j), int(k), p.ctypes.data)


def support(particle, nx, ny) -> float:
    p = _particles(particle if not isinstance(particle, dict) else [particle])
    return load().orc_support(p.ctypes.data, float(nx), float(ny))


def integrate(particle, Fx, Fy, Tz):
    p = _particles(particle if not isinstance(particle, dict) else [particle])
    out = np.zeros(1, ORC_PARTICLE_DTYPE)
    load().orc_integrate(p.ctypes.data, float(Fx), float(Fy), float(Tz), out.ctypes.data)
    return out[0]


def refill_direction(dx, dy) -> int:
    return load().orc_refill_direction(float(dx), float(dy))


def refill_node(y1, y2, y3, nvalid, uwx, uwy, Tw):
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (y1, y2, y3)]
    fh, f, g = np.empty(9), np.empty(9), np.empty(5)
    load().orc_refill_node(_dptr(a[0]), _dptr(a[1]), _dptr(a[2]), int(nvalid), float(uwx),
                           float(uwy), float(Tw), _dptr(fh), _dptr(f), _dptr(g))
    return fh, f, g
