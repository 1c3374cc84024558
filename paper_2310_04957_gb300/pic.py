"""Thin Python binding of libpic_gb300.so (include/pic.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  PyTorch supplies the CUDA stream.  If the library is missing the
import of this module fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic_gb300.so")

PIC_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOCONV", -5: "ETIMEOUT", -6: "EOVERFLOW", -7: "ENAN",
          -8: "EIO"}
PIC_EINVAL, PIC_ENOMEM, PIC_ECUDA, PIC_ENOCONV, PIC_ETIMEOUT, PIC_EOVERFLOW, PIC_ENAN, PIC_EIO = range(-1, -9, -1)
PIC_FLAG_OVERFLOW, PIC_FLAG_TIMEOUT, PIC_FLAG_NOCONV, PIC_FLAG_NAN = 0x1, 0x2, 0x4, 0x8
PIC_FP32, PIC_FP64 = 0, 1
PIC_SOLVER_PLAIN, PIC_SOLVER_MIXED, PIC_SOLVER_LEARNED, PIC_SOLVER_MG = 0, 1, 2, 3
PIC_FIELD_DIRECT, PIC_FIELD_VAHEDI = 0, 1
DIAG = {"phi": 0, "Er": 1, "Ez": 2, "chi": 3, "dep_e": 4, "dep_i": 5, "sigma": 6, "vnode": 7, "rho": 8,
        "ne_avg": 9, "ni_avg": 10, "phi_warm": 11, "phiP": 12, "phiL0": 13, "phiL1": 14, "phiL2": 15, "phiL3": 16}
DIAG_SCALARS = 100
DIAG_STORE = 101
DIAG_SOLVER = 102
DIAG_CIRCUIT = 103
DIAG_DEVICE = 0x10000  # or'ed into a selector: the buffer is device memory
NSCALARS = 49
SCALARS = ["step", "t", "U_E", "Q_E", "C_eq", "I_conv", "I_ccp", "y0", "y1", "y2", "y3", "y4", "y5", "pcg_iters",
           "pcg_relres", "numax_e", "numax_i", "pcoll_e", "pcoll_i", "absq_e_pow", "absq_e_gnd", "absq_e_surf",
           "absq_i_pow", "absq_i_gnd", "absq_i_surf", "absn_e_pow", "absn_e_gnd", "absn_e_surf", "absn_i_pow",
           "absn_i_gnd", "absn_i_surf", "coll_e_el", "coll_e_ex", "coll_e_iz", "coll_i_iso", "coll_i_cx",
           "coll_i_none", "born_e", "born_i", "ioncur_pow", "ioncur_gnd", "ioncur_surf", "i1_re", "i1_im",
           "windows", "ceq_gauss", "pcg_status", "splits_e", "splits_i"]
EXPORTS = ["pic_init", "pic_set_particles", "pic_count", "pic_get_particles", "pic_start", "pic_step",
           "pic_particle_phase", "pic_field_solve", "pic_ceq", "pic_diag", "pic_set_field", "pic_set_step",
           "pic_set_ceq", "pic_set_circuit_state", "pic_set_conv_current", "pic_circuit_run", "pic_status",
           "pic_philox", "pic_enable_timing", "pic_step_timing", "pic_strerror", "pic_destroy",
           "pic_pcg_solve_static", "pic_unet_create", "pic_unet_destroy", "pic_unet_param_count",
           "pic_unet_set_params", "pic_unet_get_params", "pic_unet_get_grads", "pic_unet_zero_grads",
           "pic_unet_forward", "pic_unet_backward", "pic_unet_adam", "pic_unet_status", "pic_conv3x3_op",
           "pic_conv3x3_op_ex", "pic_attach_unet", "pic_keep_warm", "pic_learned_pair", "pic_learned_stats",
           "pic_unet_loss_backward", "pic_learned_snapshot", "pic_batch_create", "pic_batch_step", "pic_batch_sync",
           "pic_batch_destroy", "pic_set_solver", "pic_check", "pic_set_spin_limit", "pic_save", "pic_load",
           "pic_pcg_static_result", "pic_diag_async", "pic_sync"]
STATIC_MAX_NODES = 139264


class PicError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({code})")
        self.code = code


class Config(ctypes.Structure):
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
        ("capacity", ctypes.c_int64 * 2), ("precision", ctypes.c_int32), ("solver", ctypes.c_int32),
        ("tile_r", ctypes.c_int32), ("tile_z", ctypes.c_int32), ("bin_slack", ctypes.c_double),
        ("spin_limit", ctypes.c_int64), ("weighted", ctypes.c_int32), ("split_cells", ctypes.c_int32),
        ("n_drive", ctypes.c_int32), ("drive_V", ctypes.c_double * 3), ("drive_f", ctypes.c_double * 3),
        ("drive_phase", ctypes.c_double * 3), ("field_mode", ctypes.c_int32),
    ]


class Particles(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("r", "z", "vr", "vt", "vz", "ar", "at", "az", "id", "cell", "w")]


_lib = None


def lib():
    """Load libpic_gb300.so; raise if it is missing (build it with build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libpic_gb300.so not found at {LIB_PATH}: run paper_2310_04957_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.pic_init.argtypes = [ctypes.POINTER(Config), P, ctypes.POINTER(P)]
        L.pic_set_particles.argtypes = [P, I, ctypes.c_int64, ctypes.POINTER(Particles)]
        L.pic_count.argtypes = [P, I, ctypes.POINTER(ctypes.c_int64)]
        L.pic_get_particles.argtypes = [P, I, ctypes.POINTER(Particles), ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        for n in ("pic_start", "pic_particle_phase"):
            getattr(L, n).argtypes = [P]
        L.pic_step.argtypes = [P, I]
        L.pic_field_solve.argtypes = [P, I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(D)]
        L.pic_ceq.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(D)]
        L.pic_diag.argtypes = [P, I, P, ctypes.c_size_t]
        L.pic_diag_async.argtypes = [P, I, P, ctypes.c_size_t]
        L.pic_sync.argtypes = [P]
        L.pic_set_field.argtypes = [P, I, P, ctypes.c_size_t]
        L.pic_set_step.argtypes = [P, ctypes.c_uint32]
        L.pic_set_ceq.argtypes = [P, D]
        L.pic_set_circuit_state.argtypes = [P, P]
        L.pic_set_conv_current.argtypes = [P, D]
        L.pic_circuit_run.argtypes = [P, I, P]
        L.pic_status.argtypes = [P, ctypes.POINTER(ctypes.c_uint32)]
        L.pic_philox.argtypes = [P, ctypes.c_int64, P, P, P]
        L.pic_enable_timing.argtypes = [P, I]
        L.pic_step_timing.argtypes = [P, P]
        L.pic_strerror.argtypes = [I]
        L.pic_strerror.restype = ctypes.c_char_p
        L.pic_destroy.argtypes = [P]
        L.pic_pcg_static_result.argtypes = [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(D)]
        L.pic_check.argtypes = [P]
        L.pic_set_spin_limit.argtypes = [P, ctypes.c_int64]
        L.pic_save.argtypes = [P, ctypes.c_char_p]
        L.pic_load.argtypes = [ctypes.c_char_p, P, ctypes.POINTER(P)]
        L.pic_pcg_solve_static.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, D, ctypes.c_int32, P,
                                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(D)]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(code, what):
    if code != PIC_OK:
        raise PicError(code, what)


def _check_device_out(out, n):
    import torch

    if not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() >= n):
        raise ValueError(f"needs a contiguous float64 CUDA tensor of at least {n} values")


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Discharge:
    """One discharge on the current CUDA device (wraps a pic_handle)."""

    def __init__(self, wl, precision=PIC_FP32, solver=PIC_SOLVER_PLAIN, stream=None, tile=(0, 0), bin_slack=0.0,
                 capacity=None, load=True, spin_limit=0, weighted=None):
        L = lib()
        self.wl = wl
        self.weighted = bool(wl.weighted if weighted is None else weighted)
        self.nr, self.nz = wl.nr, wl.nz
        keep = []

        def arr(a, dt):
            b = np.ascontiguousarray(a, dtype=dt)
            keep.append(b)
            return _p(b)

        c = Config()
        c.nr, c.nz, c.dr, c.dz = wl.nr, wl.nz, wl.dr, wl.dz
        c.node_kind = arr(wl.node_kind, np.int8)
        c.cell_kind = arr(wl.cell_kind, np.int8)
        c.cell_eps = arr(wl.cell_eps, np.float64)
        c.dt, c.n_gas, c.T_gas, c.m_gas = wl.dt, wl.n_gas, wl.T_gas, wl.m_gas
        c.q[:], c.m[:], c.w[:] = list(wl.q), list(wl.m), list(wl.w)
        c.n_xs = len(wl.xs_energy)
        c.xs_energy = arr(wl.xs_energy, np.float64)
        c.xs_sigma = arr(wl.xs_sigma, np.float64)
        c.thr_ex, c.thr_iz, c.B_ej = wl.thr_ex, wl.thr_iz, wl.B_ej
        c.circuit = wl.circuit
        c.circ[:] = list(wl.circ)
        c.V_src, c.f_src, c.phase_src = wl.V_src, wl.f_src, wl.phase_src
        c.n_sub, c.steps_per_rf = wl.n_sub, wl.steps_per_rf
        c.pcg_tol, c.pcg_maxit, c.ceq_refresh, c.seed = wl.pcg_tol, wl.pcg_maxit, wl.ceq_refresh, wl.seed
        cap = capacity if capacity is not None else wl.capacity
        c.capacity[:] = [int(cap[0]), int(cap[1])]
        c.precision, c.solver = precision, solver
        c.tile_r, c.tile_z = tile
        c.bin_slack = bin_slack
        c.spin_limit = spin_limit
        c.weighted = int(self.weighted)
        c.split_cells = int(wl.split_cells)
        drive = tuple(wl.drive)
        c.n_drive = len(drive)
        for k, (V, f, ph) in enumerate(drive):
            c.drive_V[k], c.drive_f[k], c.drive_phase[k] = V, f, ph
        c.field_mode = int(wl.field_mode)
        h = ctypes.c_void_p()
        _check(L.pic_init(ctypes.byref(c), _stream(stream), ctypes.byref(h)), "pic_init")
        self.h = h
        self.capacity = (int(cap[0]), int(cap[1]))
        if load:
            for s in (0, 1):
                self.set_particles(s, wl.particles[s])

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    @property
    def n_nodes(self):
        return (self.nr + 1) * (self.nz + 1)

    # -- particles
    def set_particles(self, s, P):
        cols = [np.ascontiguousarray(getattr(P, k), np.float64) for k in ("r", "z", "vr", "vt", "vz", "ar", "at", "az")]
        ids = np.ascontiguousarray(P.id, np.uint64)
        w = None if getattr(P, "w", None) is None else np.ascontiguousarray(P.w, np.float64)
        v = Particles(*[_p(x) for x in cols], _p(ids), None, None if w is None else _p(w))
        _check(lib().pic_set_particles(self.h, s, P.n, ctypes.byref(v)), "pic_set_particles")

    def count(self, s):
        n = ctypes.c_int64()
        _check(lib().pic_count(self.h, s, ctypes.byref(n)), "pic_count")
        return n.value

    def get_particles(self, s):
        n = self.count(s)
        out = {k: np.zeros(n) for k in ("r", "z", "vr", "vt", "vz", "ar", "at", "az")}
        out["id"] = np.zeros(n, np.uint64)
        out["cell"] = np.zeros(n, np.int32)
        out["w"] = np.zeros(n)
        v = Particles(*[_p(out[k]) for k in ("r", "z", "vr", "vt", "vz", "ar", "at", "az", "id", "cell", "w")])
        got = ctypes.c_int64()
        _check(lib().pic_get_particles(self.h, s, ctypes.byref(v), n, ctypes.byref(got)), "pic_get_particles")
        assert got.value == n
        return out

    # -- stepping
    def start(self):
        _check(lib().pic_start(self.h), "pic_start")

    def step(self, n=1):
        _check(lib().pic_step(self.h, n), "pic_step")

    def particle_phase(self):
        _check(lib().pic_particle_phase(self.h), "pic_particle_phase")

    def field_solve(self, mode=PIC_SOLVER_PLAIN):
        it = ctypes.c_int()
        rr = ctypes.c_double()
        st = lib().pic_field_solve(self.h, mode, ctypes.byref(it), ctypes.byref(rr))
        return st, it.value, rr.value

    def ceq(self, with_chi=False):
        c, g = ctypes.c_double(), ctypes.c_double()
        _check(lib().pic_ceq(self.h, int(with_chi), ctypes.byref(c), ctypes.byref(g)), "pic_ceq")
        return c.value, g.value

    # -- fields and scalars
    def field(self, name):
        o = np.zeros(self.n_nodes)
        _check(lib().pic_diag(self.h, DIAG[name], _p(o), o.nbytes), f"pic_diag({name})")
        return o.reshape(self.nz + 1, self.nr + 1)

    def field_to(self, name, out):
        """Enqueue the copy of a node array into `out`, a contiguous float64 CUDA tensor of
        at least n_nodes values on the handle's device (no host round trip; the copy runs
        on the handle's stream)."""
        _check_device_out(out, self.n_nodes)
        _check(lib().pic_diag(self.h, DIAG[name] | DIAG_DEVICE, ctypes.c_void_p(out.data_ptr()),
                              out.numel() * 8), f"pic_diag({name}, device)")

    def scalars_to(self, out):
        """Enqueue the scalars' copy into `out`, a contiguous float64 CUDA tensor of at least
        NSCALARS values (the handle's stream)."""
        _check_device_out(out, NSCALARS)
        _check(lib().pic_diag(self.h, DIAG_SCALARS | DIAG_DEVICE, ctypes.c_void_p(out.data_ptr()),
                              out.numel() * 8), "pic_diag(scalars, device)")

    def set_field(self, name, values):
        v = np.ascontiguousarray(values, np.float64).ravel()
        _check(lib().pic_set_field(self.h, DIAG[name], _p(v), v.size), f"pic_set_field({name})")

    def store_stats(self):
        """Per species: particles in bins, in the overflow region, capacity, overflow start."""
        o = np.zeros(8)
        _check(lib().pic_diag(self.h, DIAG_STORE, _p(o), o.nbytes), "pic_diag(store)")
        keys = ("in_bins", "overflow", "capacity", "overflow_start")
        return [dict(zip(keys, o[4 * s:4 * s + 4].astype(np.int64).tolist())) for s in (0, 1)]

    def circuit_diag(self):
        """Circuit post-processing of the last RF window (Eqs. 11-14) as a dict."""
        o = np.zeros(18)
        _check(lib().pic_diag(self.h, DIAG_CIRCUIT, _p(o), o.nbytes), "pic_diag(circuit)")
        return {"z_ccp": complex(o[0], o[1]), "z_load": complex(o[2], o[3]), "gamma": complex(o[4], o[5]),
                "gamma_abs": o[6], "p_source": o[7], "p_rs": o[8], "p_series": o[9], "p_stray": o[10],
                "p_ccp": o[11], "p_forward": o[12], "p_ref": o[13], "u1": complex(o[14], o[15]),
                "u_dc": o[16], "i_dc": o[17]}

    def solver_state(self):
        """Multigrid solves counter, rebuild period, last iterations, outer steps, status."""
        o = np.zeros(5)
        _check(lib().pic_diag(self.h, DIAG_SOLVER, _p(o), o.nbytes), "pic_diag(solver)")
        return dict(zip(("mg_solves", "rebuild_every", "iters", "outer", "status"), o.astype(np.int64).tolist()))

    def scalars(self):
        o = np.zeros(NSCALARS)
        _check(lib().pic_diag(self.h, DIAG_SCALARS, _p(o), o.nbytes), "pic_diag(scalars)")
        return dict(zip(SCALARS, o.tolist()))

    def scalars_async(self, out):
        """Enqueue the read of the scalars at this point of the stream into `out` (a
        C-contiguous float64 array of at least NSCALARS values, kept alive by the
        caller; page-locked memory for a copy that does not wait). The values are
        there after sync() or any synchronising call."""
        if out.dtype != np.float64 or out.size < NSCALARS or not out.flags.c_contiguous:
            raise ValueError("scalars_async needs a C-contiguous float64 array of NSCALARS values")
        _check(lib().pic_diag_async(self.h, DIAG_SCALARS, _p(out), out.nbytes), "pic_diag_async")

    def sync(self):
        _check(lib().pic_sync(self.h), "pic_sync")

    def set_step(self, n):
        _check(lib().pic_set_step(self.h, n), "pic_set_step")

    def set_ceq(self, c):
        _check(lib().pic_set_ceq(self.h, c), "pic_set_ceq")

    def set_circuit_state(self, y):
        y = np.zeros(6) if y is None else np.ascontiguousarray(y, np.float64)
        _check(lib().pic_set_circuit_state(self.h, _p(y)), "pic_set_circuit_state")

    def set_conv_current(self, i):
        _check(lib().pic_set_conv_current(self.h, i), "pic_set_conv_current")

    def circuit_run(self, n):
        U = np.zeros(n)
        _check(lib().pic_circuit_run(self.h, n, _p(U)), "pic_circuit_run")
        return U

    def status(self):
        f = ctypes.c_uint32()
        _check(lib().pic_status(self.h, ctypes.byref(f)), "pic_status")
        return f.value

    def check(self):
        """PIC_OK or the code of the most severe accumulated status bit (not cleared)."""
        return lib().pic_check(self.h)

    def set_spin_limit(self, cycles):
        _check(lib().pic_set_spin_limit(self.h, int(cycles)), "pic_set_spin_limit")

    def save(self, path):
        _check(lib().pic_save(self.h, os.fsencode(path)), "pic_save")

    @classmethod
    def load(cls, path, wl, stream=None):
        """Restore a discharge written by save(); `wl` (the workload it was made
        from) only supplies the grid shape and inputs for reference."""
        h = ctypes.c_void_p()
        _check(lib().pic_load(os.fsencode(path), _stream(stream), ctypes.byref(h)), "pic_load")
        d = cls.__new__(cls)
        d.wl, d.nr, d.nz, d.h = wl, wl.nr, wl.nz, h
        d.capacity = tuple(wl.capacity)
        d.weighted = bool(wl.weighted)
        return d

    def philox(self, ctr, key):
        ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
        key = np.ascontiguousarray(key, np.uint32).reshape(-1, 2)
        out = np.zeros_like(ctr)
        _check(lib().pic_philox(self.h, ctr.shape[0], _p(ctr), _p(key), _p(out)), "pic_philox")
        return out

    def enable_timing(self, on=True):
        _check(lib().pic_enable_timing(self.h, int(on)), "pic_enable_timing")

    def step_timing(self):
        o = np.zeros(7)
        _check(lib().pic_step_timing(self.h, _p(o)), "pic_step_timing")
        return o

    # -- learned field solve
    def attach_unet(self, net, maxit=200, smooth=0, finish=PIC_SOLVER_PLAIN):
        """Use `net` (a UNet of H = nz, W = nr) in PIC_SOLVER_LEARNED solves: at most
        maxit network applications, then `finish` confirms / completes the solve."""
        L = lib()
        L.pic_attach_unet.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _check(L.pic_attach_unet(self.h, net.h if net is not None else None, maxit, smooth, finish),
               "pic_attach_unet")
        self._net = net

    def set_solver(self, solver):
        _check(lib().pic_set_solver(self.h, solver), "pic_set_solver")

    def keep_warm(self, on=True):
        _check(lib().pic_keep_warm(self.h, int(on)), "pic_keep_warm")

    def learned_pair(self, in3_ptr, target_ptr, source=0):
        """Training pair of the last solve into device FP32 buffers; returns the scale s.
        source 0: from the warm start; 1: from the kept learned iterate."""
        L = lib()
        L.pic_learned_pair.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]
        s = ctypes.c_double()
        _check(L.pic_learned_pair(self.h, source, in3_ptr, target_ptr, ctypes.byref(s)), "pic_learned_pair")
        return s.value

    def learned_snapshot(self, k):
        _check(lib().pic_learned_snapshot(self.h, k), "pic_learned_snapshot")

    def learned_stats(self):
        o = np.zeros(4)
        _check(lib().pic_learned_stats(self.h, _p(o)), "pic_learned_stats")
        return o


def pcg_solve_static(nr, nz, node_kind, Gr, Gz, qrhs, phi, tol, maxit, stream=None, wait=True):
    """Call pic_pcg_solve_static on caller-owned device arrays (raw device pointers as ints).

    The library allocates nothing for this solve.  wait=True: returns (status,
    iterations, relative residual) after synchronising the stream; wait=False:
    only enqueues it (NULL outputs) and returns (status of the enqueue, None, None);
    pcg_static_result() reads the outcome later."""
    it = ctypes.c_int32()
    rr = ctypes.c_double()
    outs = (ctypes.byref(it), ctypes.byref(rr)) if wait else (None, None)
    st = lib().pic_pcg_solve_static(nr, nz, ctypes.c_void_p(node_kind), ctypes.c_void_p(Gr), ctypes.c_void_p(Gz),
                                    ctypes.c_void_p(qrhs), ctypes.c_void_p(phi), tol, maxit, _stream(stream), *outs)
    return (st, it.value, rr.value) if wait else (st, None, None)


def pcg_static_result(stream=None):
    """(status, iterations, relative residual) of the last pic_pcg_solve_static call."""
    it = ctypes.c_int32()
    rr = ctypes.c_double()
    st = lib().pic_pcg_static_result(_stream(stream), ctypes.byref(it), ctypes.byref(rr))
    return st, it.value, rr.value


class UNet:
    """The learned preconditioner's network on the current device (wraps pic_unet)."""

    def __init__(self, H, W, stream=None):
        L = lib()
        P = ctypes.c_void_p
        for name, args in (("pic_unet_create", [ctypes.c_int, ctypes.c_int, P, ctypes.POINTER(P)]),
                           ("pic_unet_destroy", [P]), ("pic_unet_param_count", [P, ctypes.POINTER(ctypes.c_int64)]),
                           ("pic_unet_set_params", [P, P, ctypes.c_int64]), ("pic_unet_get_params", [P, P, ctypes.c_int64]),
                           ("pic_unet_get_grads", [P, P, ctypes.c_int64]), ("pic_unet_zero_grads", [P]),
                           ("pic_unet_forward", [P, P, P]), ("pic_unet_backward", [P, P]),
                           ("pic_unet_adam", [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int]),
                           ("pic_unet_status", [P, ctypes.POINTER(ctypes.c_int)])):
            getattr(L, name).argtypes = args
        h = ctypes.c_void_p()
        _check(L.pic_unet_create(H, W, _stream(stream), ctypes.byref(h)), "pic_unet_create")
        self.h, self.H, self.W = h, H, W
        n = ctypes.c_int64()
        _check(L.pic_unet_param_count(h, ctypes.byref(n)), "pic_unet_param_count")
        self.nparams = n.value

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.pic_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        _check(lib().pic_unet_set_params(self.h, _p(p), p.size), "pic_unet_set_params")

    def get_params(self):
        o = np.zeros(self.nparams, np.float32)
        _check(lib().pic_unet_get_params(self.h, _p(o), o.size), "pic_unet_get_params")
        return o

    def get_grads(self):
        o = np.zeros(self.nparams, np.float32)
        _check(lib().pic_unet_get_grads(self.h, _p(o), o.size), "pic_unet_get_grads")
        return o

    def zero_grads(self):
        _check(lib().pic_unet_zero_grads(self.h), "pic_unet_zero_grads")

    def forward(self, inp_ptr, out_ptr):
        """inp_ptr: device FP32 [3][H*W]; out_ptr: device FP32 [H*W] (raw pointers)."""
        _check(lib().pic_unet_forward(self.h, ctypes.c_void_p(inp_ptr), ctypes.c_void_p(out_ptr)), "pic_unet_forward")

    def backward(self, gout_ptr):
        _check(lib().pic_unet_backward(self.h, ctypes.c_void_p(gout_ptr)), "pic_unet_backward")

    def loss_backward(self, in3_ptr, target_ptr, loss_ptr=0):
        """Relative L2 loss of the last forward against the target over free pixels;
        backpropagates it and adds it to the device float at loss_ptr (if nonzero)."""
        L = lib()
        L.pic_unet_loss_backward.argtypes = [ctypes.c_void_p] * 4
        _check(L.pic_unet_loss_backward(self.h, ctypes.c_void_p(in3_ptr), ctypes.c_void_p(target_ptr),
                                        ctypes.c_void_p(loss_ptr) if loss_ptr else None), "pic_unet_loss_backward")

    def adam(self, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().pic_unet_adam(self.h, lr, beta1, beta2, eps, t), "pic_unet_adam")

    def status(self):
        e = ctypes.c_int()
        _check(lib().pic_unet_status(self.h, ctypes.byref(e)), "pic_unet_status")
        return e.value


def conv3x3_op(op, H, W, inp_ptr, Cin, w_ptr, bias_ptr, out_ptr, Cout, stream=None, tile_n=0, tile_mma=0):
    """Call pic_conv3x3_op_ex on raw device pointers; returns the status code.
    tile_n / tile_mma force a tiling (0 = automatic, tile_n = -1 = gather kernel)."""
    L = lib()
    P = ctypes.c_void_p
    I = ctypes.c_int
    L.pic_conv3x3_op_ex.argtypes = [I, I, I, P, I, P, P, P, I, I, I, P]
    return L.pic_conv3x3_op_ex(op, H, W, P(inp_ptr), Cin, P(w_ptr), P(bias_ptr) if bias_ptr else None, P(out_ptr),
                               Cout, tile_n, tile_mma, _stream(stream))


class Batch:
    """Independent discharges stepped together in one graph per step (wraps pic_batch)."""

    def __init__(self, discharges):
        L = lib()
        L.pic_batch_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
        L.pic_batch_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.pic_batch_sync.argtypes = [ctypes.c_void_p]
        L.pic_batch_destroy.argtypes = [ctypes.c_void_p]
        self.discharges = list(discharges)
        arr = (ctypes.c_void_p * len(self.discharges))(*[d.h.value for d in self.discharges])
        h = ctypes.c_void_p()
        _check(L.pic_batch_create(arr, len(self.discharges), ctypes.byref(h)), "pic_batch_create")
        self.h = h

    def step(self, n=1):
        _check(lib().pic_batch_step(self.h, n), "pic_batch_step")

    def sync(self):
        _check(lib().pic_batch_sync(self.h), "pic_batch_sync")

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.pic_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()
