"""ctypes binding of the FP64 CPU oracle (oracle/pic_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by bench.py's cpu_baseline / reference arm, never by the product package.
It takes the seeded inputs as plain attributes of a workload object and
shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

FIELD = {"phi": 0, "Er": 1, "Ez": 2, "chi": 3, "dep_e": 4, "dep_i": 5, "sigma": 6, "vnode": 7, "rho": 8,
         "ne_avg": 9, "ni_avg": 10, "phiP": 11, "phiL0": 12, "phiL1": 13, "phiL2": 14, "phiL3": 15}


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain -O2, IEEE, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pic_oracle.h"))):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


class Setup(ctypes.Structure):
    _fields_ = [
        ("nr", ctypes.c_int32), ("nz", ctypes.c_int32), ("dr", ctypes.c_double), ("dz", ctypes.c_double),
        ("node_kind", ctypes.c_void_p), ("cell_kind", ctypes.c_void_p), ("cell_eps", ctypes.c_void_p),
        ("dt", ctypes.c_double), ("n_gas", ctypes.c_double), ("T_gas", ctypes.c_double), ("m_gas", ctypes.c_double),
        ("q", ctypes.c_double * 2), ("m", ctypes.c_double * 2), ("w", ctypes.c_double * 2),
        ("n_xs", ctypes.c_int32), ("xs_energy", ctypes.c_void_p), ("xs_sigma", ctypes.c_void_p),
        ("thr_ex", ctypes.c_double), ("thr_iz", ctypes.c_double), ("B_ej", ctypes.c_double),
        ("circuit", ctypes.c_int32), ("circ", ctypes.c_double * 8),
        ("V_src", ctypes.c_double), ("f_src", ctypes.c_double), ("phase_src", ctypes.c_double),
        ("n_sub", ctypes.c_int32), ("steps_per_rf", ctypes.c_int32), ("pcg_tol", ctypes.c_double),
        ("pcg_maxit", ctypes.c_int32), ("ceq_refresh", ctypes.c_int32), ("seed", ctypes.c_uint32),
        ("capacity", ctypes.c_int64 * 2), ("split_cells", ctypes.c_int32),
        ("n_drive", ctypes.c_int32), ("drive_V", ctypes.c_double * 3), ("drive_f", ctypes.c_double * 3),
        ("drive_phase", ctypes.c_double * 3), ("field_mode", ctypes.c_int32),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(Setup), ctypes.POINTER(P)]
        L.orc_destroy.argtypes = [P]
        L.orc_set_particles.argtypes = [P, ctypes.c_int, ctypes.c_int64] + [P] * 10
        L.orc_count.argtypes = [P, ctypes.c_int]
        L.orc_count.restype = ctypes.c_int64
        L.orc_get_particles.argtypes = [P, ctypes.c_int] + [P] * 11
        for name in ("orc_get_field", "orc_set_field", "orc_get_operator"):
            getattr(L, name).argtypes = [P, ctypes.c_int, P]
        L.orc_set_step.argtypes = [P, ctypes.c_uint32]
        for name in ("orc_particle_phase", "orc_deposit_only", "orc_assemble", "orc_efield", "orc_circuit_advance",
                     "orc_init_fields"):
            getattr(L, name).argtypes = [P]
        L.orc_field_solve.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.orc_solve_tol.argtypes = [P, ctypes.c_double, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.orc_ceq.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.orc_set_ceq.argtypes = [P, ctypes.c_double]
        L.orc_set_conv_current.argtypes = [P, ctypes.c_double]
        L.orc_set_circuit_state.argtypes = [P, P]
        L.orc_step.argtypes = [P, ctypes.c_int]
        L.orc_circuit_run.argtypes = [P, ctypes.c_int, P]
        L.orc_scalars.argtypes = [P, P, ctypes.c_int]
        L.orc_philox.argtypes = [P, P, P]
        L.orc_xs.argtypes = [P, ctypes.c_int, ctypes.c_double]
        L.orc_xs.restype = ctypes.c_double
        L.orc_scatter_cos.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_scatter_cos.restype = ctypes.c_double
        L.orc_turn.argtypes = [P, ctypes.c_double, ctypes.c_double]
        L.orc_trace.argtypes = [P, ctypes.c_int, P]
        L.orc_circuit_diag.argtypes = [P, P]
        L.orc_child_ids.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64, P, P]
        L.orc_split_ids.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int64, P, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


SCALARS = ["step", "t", "U_E", "Q_E", "C_eq", "I_conv", "I_ccp", "y0", "y1", "y2", "y3", "y4", "y5", "pcg_iters",
           "pcg_relres", "numax_e", "numax_i", "pcoll_e", "pcoll_i", "absq_e_pow", "absq_e_gnd", "absq_e_surf",
           "absq_i_pow", "absq_i_gnd", "absq_i_surf", "absn_e_pow", "absn_e_gnd", "absn_e_surf", "absn_i_pow",
           "absn_i_gnd", "absn_i_surf", "coll_e_el", "coll_e_ex", "coll_e_iz", "coll_i_iso", "coll_i_cx",
           "coll_i_none", "born_e", "born_i", "ioncur_pow", "ioncur_gnd", "ioncur_surf", "i1_re", "i1_im",
           "windows", "ceq_gauss", "pcg_status", "splits_e", "splits_i"]


def philox(ctr, key):
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().orc_philox(_p(c), _p(k), _p(o))
    return o


CIRCUIT_KEYS = ("z_ccp", "z_load", "gamma", "gamma_abs", "p_source", "p_rs", "p_series", "p_stray", "p_ccp",
                "p_forward", "p_ref", "u1")


def circuit_dict(o):
    return {"z_ccp": complex(o[0], o[1]), "z_load": complex(o[2], o[3]), "gamma": complex(o[4], o[5]),
            "gamma_abs": o[6], "p_source": o[7], "p_rs": o[8], "p_series": o[9], "p_stray": o[10], "p_ccp": o[11],
            "p_forward": o[12], "p_ref": o[13], "u1": complex(o[14], o[15]), "u_dc": o[16], "i_dc": o[17]}


def child_ids(step, seed, parents):
    """[n, 2] ids of the electron and ion an ionization of each parent creates in `step`."""
    p = np.ascontiguousarray(parents, np.uint64)
    out = np.zeros((len(p), 2), np.uint64)
    lib().orc_child_ids(step, seed, len(p), _p(p), _p(out))
    return out


def split_ids(step, seed, parents):
    """Id of the second half of each parent if it splits in `step`."""
    p = np.ascontiguousarray(parents, np.uint64)
    out = np.zeros(len(p), np.uint64)
    lib().orc_split_ids(step, seed, len(p), _p(p), _p(out))
    return out


class Oracle:
    """One oracle discharge built from a workload's input arrays."""

    def __init__(self, wl, capacity=None, set_particles=True):
        L = lib()
        self.wl = wl
        self.nr, self.nz = wl.nr, wl.nz
        self._keep = []

        def arr(a, dt):
            b = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(b)
            return _p(b)

        s = Setup()
        s.nr, s.nz, s.dr, s.dz = wl.nr, wl.nz, wl.dr, wl.dz
        s.node_kind = arr(wl.node_kind, np.int8)
        s.cell_kind = arr(wl.cell_kind, np.int8)
        s.cell_eps = arr(wl.cell_eps, np.float64)
        s.dt, s.n_gas, s.T_gas, s.m_gas = wl.dt, wl.n_gas, wl.T_gas, wl.m_gas
        s.q[:] = list(wl.q)
        s.m[:] = list(wl.m)
        s.w[:] = list(wl.w)
        s.n_xs = len(wl.xs_energy)
        s.xs_energy = arr(wl.xs_energy, np.float64)
        s.xs_sigma = arr(wl.xs_sigma, np.float64)
        s.thr_ex, s.thr_iz, s.B_ej = wl.thr_ex, wl.thr_iz, wl.B_ej
        s.circuit = wl.circuit
        s.circ[:] = list(wl.circ)
        s.V_src, s.f_src, s.phase_src = wl.V_src, wl.f_src, wl.phase_src
        s.n_sub, s.steps_per_rf = wl.n_sub, wl.steps_per_rf
        s.pcg_tol, s.pcg_maxit, s.ceq_refresh, s.seed = wl.pcg_tol, wl.pcg_maxit, wl.ceq_refresh, wl.seed
        cap = capacity if capacity is not None else wl.capacity
        s.capacity[:] = [int(cap[0]), int(cap[1])]
        s.split_cells = int(getattr(wl, "split_cells", 0))
        drive = tuple(getattr(wl, "drive", ()))
        s.n_drive = len(drive)
        for k, (V, f, ph) in enumerate(drive):
            s.drive_V[k], s.drive_f[k], s.drive_phase[k] = V, f, ph
        s.field_mode = int(getattr(wl, "field_mode", 0))
        h = ctypes.c_void_p()
        st = L.orc_create(ctypes.byref(s), ctypes.byref(h))
        if st != 0:
            raise RuntimeError(f"orc_create failed: {st}")
        self.h = h
        self._keep = []
        if set_particles:
            for spc in (0, 1):
                self.set_particles(spc, wl.particles[spc])

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.orc_destroy(h)
            self.h = None

    @property
    def n_nodes(self):
        return (self.nr + 1) * (self.nz + 1)

    def set_particles(self, spc, P):
        a = [np.ascontiguousarray(getattr(P, k), np.float64) for k in ("r", "z", "vr", "vt", "vz", "ar", "at", "az")]
        ids = np.ascontiguousarray(P.id, np.uint64)
        w = getattr(P, "w", None)
        w = None if w is None else np.ascontiguousarray(w, np.float64)
        st = lib().orc_set_particles(self.h, spc, P.n, *[_p(x) for x in a], _p(ids), None if w is None else _p(w))
        if st != 0:
            raise RuntimeError(f"orc_set_particles failed: {st}")

    def count(self, spc):
        return int(lib().orc_count(self.h, spc))

    def get_particles(self, spc):
        n = self.count(spc)
        out = {k: np.zeros(n) for k in ("r", "z", "vr", "vt", "vz", "ar", "at", "az")}
        out["id"] = np.zeros(n, np.uint64)
        out["cell"] = np.zeros(n, np.int32)
        out["w"] = np.zeros(n)
        keys = ("r", "z", "vr", "vt", "vz", "ar", "at", "az", "id", "cell", "w")
        lib().orc_get_particles(self.h, spc, *[_p(out[k]) for k in keys])
        return out

    def field(self, name):
        o = np.zeros(self.n_nodes)
        st = lib().orc_get_field(self.h, FIELD[name], _p(o))
        if st:
            raise RuntimeError(st)
        return o.reshape(self.nz + 1, self.nr + 1)

    def set_field(self, name, values):
        v = np.ascontiguousarray(values, np.float64).ravel()
        assert v.size == self.n_nodes
        st = lib().orc_set_field(self.h, FIELD[name], _p(v))
        if st:
            raise RuntimeError(st)

    def operator(self):
        gr = np.zeros((self.nz + 1) * self.nr)
        gz = np.zeros(self.nz * (self.nr + 1))
        lib().orc_get_operator(self.h, 0, _p(gr))
        lib().orc_get_operator(self.h, 1, _p(gz))
        return gr.reshape(self.nz + 1, self.nr), gz.reshape(self.nz, self.nr + 1)

    def set_step(self, n):
        lib().orc_set_step(self.h, n)

    def _check(self, st, what):
        if st != 0:
            raise RuntimeError(f"{what} failed with status {st}")

    def particle_phase(self):
        self._check(lib().orc_particle_phase(self.h), "particle_phase")

    def deposit_only(self):
        self._check(lib().orc_deposit_only(self.h), "deposit_only")

    def assemble(self):
        self._check(lib().orc_assemble(self.h), "assemble")

    def field_solve(self):
        it = ctypes.c_int()
        rr = ctypes.c_double()
        st = lib().orc_field_solve(self.h, ctypes.byref(it), ctypes.byref(rr))
        return st, it.value, rr.value

    def solve_tol(self, tol):
        it = ctypes.c_int()
        rr = ctypes.c_double()
        st = lib().orc_solve_tol(self.h, tol, ctypes.byref(it), ctypes.byref(rr))
        return st, it.value, rr.value

    def efield(self):
        lib().orc_efield(self.h)

    def ceq(self, with_chi=False):
        c = ctypes.c_double()
        g = ctypes.c_double()
        st = lib().orc_ceq(self.h, int(with_chi), ctypes.byref(c), ctypes.byref(g))
        self._check(st, "ceq")
        return c.value, g.value

    def set_ceq(self, c):
        lib().orc_set_ceq(self.h, c)

    def set_conv_current(self, i):
        lib().orc_set_conv_current(self.h, i)

    def set_circuit_state(self, y):
        y = np.zeros(6) if y is None else np.ascontiguousarray(y, np.float64)
        lib().orc_set_circuit_state(self.h, _p(y))

    def circuit_advance(self):
        lib().orc_circuit_advance(self.h)

    def circuit_run(self, n):
        U = np.zeros(n)
        lib().orc_circuit_run(self.h, n, _p(U))
        return U

    def init_fields(self):
        self._check(lib().orc_init_fields(self.h), "init_fields")

    def step(self, n=1):
        self._check(lib().orc_step(self.h, n), "step")

    def scalars(self):
        o = np.zeros(len(SCALARS))
        lib().orc_scalars(self.h, _p(o), len(SCALARS))
        return dict(zip(SCALARS, o.tolist()))

    def xs(self, proc, E):
        return lib().orc_xs(self.h, proc, float(E))

    def circuit_diag(self):
        """Circuit post-processing of the last closed window (Eqs. 11-14), as a dict."""
        o = np.zeros(18)
        lib().orc_circuit_diag(self.h, _p(o))
        return circuit_dict(o)

    def trace(self, enable):
        """Decision-margin tracing: enable=True resets and starts recording,
        False stops, None only reads.  Returns the margins recorded so far:
        (random-number / energy thresholds, relative; position tests, cell
        units; predictor rotation conditioning)."""
        out = np.zeros(3)
        lib().orc_trace(self.h, -1 if enable is None else int(bool(enable)), _p(out))
        return tuple(out.tolist())


def scatter_cos(E, R):
    return lib().orc_scatter_cos(float(E), float(R))


def turn(c, cc, phi):
    v = np.ascontiguousarray(c, np.float64).copy()
    lib().orc_turn(_p(v), float(cc), float(phi))
    return v
