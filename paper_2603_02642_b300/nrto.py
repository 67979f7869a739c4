"""ctypes binding of libnrto (include/nrto.h).  Argument marshalling only: every step of the
solver runs in the library's CUDA kernels.  `load()` raises if the shared library is missing;
there is no CPU fallback."""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("NRTO_LIB", os.path.join(HERE, "libnrto.so"))

PREC_FP64, PREC_MIXED = 0, 1
NSTAT = 15   # NRTO_NSTAT
NMAPPING = 4  # NRTO_NMAPPING
SOLVER_DR, SOLVER_FULLADMM, SOLVER_FULLADMM_AW = 0, 1, 2

(F_XHAT, F_UHAT, F_A, F_B, F_G0, F_BHAT, F_BVEC, F_LAMNU, F_K, F_DU, F_P, F_PT, F_LAMP, F_GM, F_KACC,
 F_DX, F_SCAL, F_STATS, F_LAMW, F_LAME, F_S) = range(21)

STATUS = {0: "OK", 1: "INVALID", 2: "CUDA", 3: "NOT_CONVERGED", 4: "NUMERIC", 5: "TIMEOUT", 6: "STATE"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


# nrto_problem_desc.  The `const double*` members are declared as void pointers (same size and
# alignment) so that the binding can store array addresses as plain integers.
_vp = C.c_void_p


class ProblemDesc(C.Structure):
    _fields_ = [("dyn", C.c_int), ("nx", C.c_int), ("nu", C.c_int), ("T", C.c_int), ("dt", C.c_double),
                ("dyn_params", _vp), ("n_dyn_params", C.c_int),
                ("x0", _vp), ("x_goal", _vp), ("u_init", _vp), ("u_ref", _vp), ("Sigma", _vp),
                ("tau", C.c_double), ("Qx", _vp), ("Ru", _vp), ("RK", _vp),
                ("n_obs", C.c_int), ("obs_dim", C.c_int), ("obs_center", _vp), ("obs_radius", _vp),
                ("n_link", C.c_int), ("link_spheres", _vp),
                ("u_lo", _vp), ("u_hi", _vp), ("x_lo", _vp), ("x_hi", _vp)]


class SolverOpts(C.Structure):
    _fields_ = [("solver", C.c_int), ("rho", C.c_double), ("alpha", C.c_double), ("r_chi", C.c_double),
                ("sigma", C.c_double), ("eps_p", C.c_double), ("eps_d", C.c_double), ("eps_dr", C.c_double),
                ("max_inner", C.c_int), ("max_dr", C.c_int), ("check", C.c_int),
                ("r0", C.c_double), ("r_min", C.c_double), ("w_p", C.c_double),
                ("adapt_every", C.c_int), ("adapt_mu", C.c_double), ("adapt_tau", C.c_double),
                ("rho_min", C.c_double), ("rho_max", C.c_double),
                ("stall_every", C.c_int), ("stall_ratio", C.c_double), ("warm_fallback", C.c_int),
                ("carry", C.c_int), ("max_inner_final", C.c_int),
                ("kv_pcg_iters", C.c_int), ("kv_pcg_tol", C.c_double), ("stall_budget", C.c_double)]


class InstanceInfo(C.Structure):
    _fields_ = [("nx", C.c_int), ("nu", C.c_int), ("T", C.c_int), ("n_rows", C.c_int),
                ("n_state_rows", C.c_int), ("n_control_rows", C.c_int),
                ("n_entries", C.c_longlong), ("n_entries_state", C.c_longlong)]


class SocpOut(C.Structure):
    _fields_ = [("du", _dp), ("K", _dp), ("p", _dp), ("ptilde", _dp), ("iters", _ip),
                ("r_p", _dp), ("r_d", _dp), ("status", _ip)]


_LIB = None


def load():
    """Load libnrto.so (built by `paper_2603_02642_b300.build.build()`)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libnrto.so not found at {LIB_PATH}; run paper_2603_02642_b300/build.py")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    lib.nrto_problem_create.argtypes = [C.POINTER(ProblemDesc), C.c_int, C.c_int, C.c_void_p, C.POINTER(P)]
    lib.nrto_problem_destroy.argtypes = [P]
    lib.nrto_problem_info.argtypes = [P, C.c_int, C.POINTER(InstanceInfo)]
    lib.nrto_problem_update.argtypes = [P, C.POINTER(ProblemDesc), C.c_int]
    lib.nrto_linearize.argtypes = [P, _dp]
    lib.nrto_set_trust_radius.argtypes = [P, _dp]
    lib.nrto_solve_socp.argtypes = [P, C.POINTER(SolverOpts), C.POINTER(SocpOut)]
    lib.nrto_outer_step.argtypes = [P, C.POINTER(SolverOpts), _ip]
    lib.nrto_solve.argtypes = [P, C.POINTER(SolverOpts), C.c_int, _dp, _dp, _dp]
    lib.nrto_set_warm_start.argtypes = [P, _dp, _dp, _dp]
    lib.nrto_export.argtypes = [P, C.c_int, C.c_int, _dp, C.c_longlong]
    lib.nrto_import.argtypes = [P, C.c_int, C.c_int, _dp, C.c_longlong]
    lib.nrto_profile.argtypes = [P, C.c_int, _dp, C.POINTER(C.c_longlong)]
    lib.nrto_phase_cycles.argtypes = [P, C.POINTER(C.c_longlong), C.c_int]
    lib.nrto_phase_cycles.restype = C.c_int
    lib.nrto_solve_noalloc.argtypes = [C.POINTER(ProblemDesc), C.c_int, C.c_int, C.POINTER(SolverOpts), C.c_int,
                                       C.c_void_p, _dp, _dp, _dp]
    _fp = C.POINTER(C.c_float)
    lib.nrto_mlp_create.argtypes = [C.POINTER(C.c_int), C.c_int, C.c_int, C.c_void_p, C.POINTER(P)]
    lib.nrto_mlp_destroy.argtypes = [P]
    lib.nrto_mlp_num_params.argtypes = [P]
    lib.nrto_mlp_num_params.restype = C.c_longlong
    lib.nrto_mlp_set_params.argtypes = [P, _fp]
    lib.nrto_mlp_get_params.argtypes = [P, _fp]
    lib.nrto_mlp_forward.argtypes = [P, _fp, C.c_int, _fp]
    lib.nrto_mlp_train_step.argtypes = [P, _fp, _fp, _fp, C.c_int, C.c_float, _dp, _fp]
    lib.nrto_set_warm_start_from_network.argtypes = [P, P, C.POINTER(C.c_float), _ip, C.c_int, C.c_int, C.c_int]
    lib.nrto_set_warm_start_from_network.restype = C.c_int
    lib.nrto_mlp_profile.argtypes = [P, C.c_int, _dp, _dp, C.POINTER(C.c_longlong)]
    lib.nrto_mlp_profile.restype = C.c_int
    lib.nrto_mlp_kernel_launches.argtypes = [P]
    lib.nrto_mlp_kernel_launches.restype = C.c_longlong
    lib.nrto_set_launch_mapping.argtypes = [P, C.c_int]
    lib.nrto_set_launch_mapping.restype = C.c_int
    lib.nrto_autotune.argtypes = [P, C.POINTER(SolverOpts), C.c_int, C.c_int, _dp, _ip]
    lib.nrto_autotune.restype = C.c_int
    lib.nrto_set_graph.argtypes = [P, C.c_int]
    lib.nrto_set_graph.restype = C.c_int
    lib.nrto_graph_info.argtypes = [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    lib.nrto_graph_info.restype = C.c_int
    lib.nrto_get_stats.argtypes = [P, _dp, C.c_int]
    lib.nrto_get_stats.restype = C.c_int
    lib.nrto_set_warm_start_lifted.argtypes = [P, _dp, _dp, _dp, _dp, _dp]
    lib.nrto_set_warm_start_lifted.restype = C.c_int
    lib.nrto_set_warm_start_from_network_lifted.argtypes = [P, P, C.POINTER(C.c_float), _ip, _ip]
    lib.nrto_set_warm_start_from_network_lifted.restype = C.c_int
    lib.nrto_monte_carlo.argtypes = [P, _dp, C.c_int, C.c_int, C.c_ulonglong, C.c_double, _ip, _dp]
    lib.nrto_monte_carlo.restype = C.c_int
    lib.nrto_kernel_launches.argtypes = [P]
    lib.nrto_kernel_launches.restype = C.c_longlong
    lib.nrto_selftest_bounded_wait.argtypes = [C.c_void_p, _ip, C.POINTER(C.c_longlong)]
    lib.nrto_selftest_bounded_wait.restype = C.c_int
    lib.nrto_last_error.restype = C.c_char_p
    for name in ["nrto_problem_create", "nrto_problem_destroy", "nrto_problem_info", "nrto_problem_update",
                 "nrto_linearize", "nrto_set_trust_radius", "nrto_solve_socp", "nrto_outer_step", "nrto_solve",
                 "nrto_set_warm_start", "nrto_export", "nrto_import", "nrto_profile", "nrto_solve_noalloc",
                 "nrto_mlp_create", "nrto_mlp_destroy", "nrto_mlp_set_params", "nrto_mlp_get_params",
                 "nrto_mlp_forward", "nrto_mlp_train_step"]:
        getattr(lib, name).restype = C.c_int
    _LIB = lib
    return lib


class NrtoError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _check(code, allow=()):
    if code != 0 and code not in allow:
        raise NrtoError(code, load().nrto_last_error().decode())
    return code


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


@dataclass
class Options:
    solver: int = SOLVER_FULLADMM
    rho: float = 10.0
    alpha: float = 0.9
    r_chi: float = 1.0
    sigma: float = 1.0
    eps_p: float = 1e-4
    eps_d: float = 1e-4
    eps_dr: float = 1e-4
    max_inner: int = 500
    max_dr: int = 500
    check: int = 1
    r0: float = 2.0
    r_min: float = 1e-3
    w_p: float = 10.0
    adapt_every: int = 0
    adapt_mu: float = 10.0
    adapt_tau: float = 2.0
    rho_min: float = 1e-3
    rho_max: float = 1e3
    stall_every: int = 0
    stall_ratio: float = 0.9
    warm_fallback: int = 0
    carry: int = 0
    max_inner_final: int = 0
    kv_pcg_iters: int = 0
    kv_pcg_tol: float = 0.05
    stall_budget: float = 0.0

    def c(self) -> SolverOpts:
        return SolverOpts(self.solver, self.rho, self.alpha, self.r_chi, self.sigma, self.eps_p, self.eps_d,
                          self.eps_dr, self.max_inner, self.max_dr, self.check, self.r0, self.r_min, self.w_p,
                          self.adapt_every, self.adapt_mu, self.adapt_tau, self.rho_min, self.rho_max,
                          self.stall_every, self.stall_ratio, self.warm_fallback, self.carry,
                          self.max_inner_final, self.kv_pcg_iters, self.kv_pcg_tol, self.stall_budget)


_ZERO1 = np.zeros(1)
_ZERO5 = np.zeros(5)


def _desc(inst, keep):
    def adr(a):
        # address of a C-contiguous float64 copy (the array itself when it already is one)
        if not (type(a) is np.ndarray and a.dtype == np.float64 and a.flags.c_contiguous):
            a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
        keep.append(a)
        return a.ctypes.data
    is_arm = inst.kind == 2
    return ProblemDesc(
        inst.kind, inst.nx, inst.nu, inst.T, inst.dt,
        adr(inst.dyn_params if inst.dyn_params.size else _ZERO1), int(inst.dyn_params.size),
        adr(inst.x0), adr(inst.x_goal), adr(inst.u_init), adr(inst.u_ref), adr(inst.Sigma),
        inst.tau, adr(inst.Qx), adr(inst.Ru), adr(inst.RK),
        inst.n_obs, inst.obs_dim,
        adr(inst.obs_center if inst.n_obs else _ZERO1), adr(inst.obs_radius if inst.n_obs else _ZERO1),
        int(inst.link_spheres.shape[0]) if is_arm else 0,
        adr(inst.link_spheres if is_arm and inst.link_spheres.size else _ZERO5),
        adr(inst.u_lo), adr(inst.u_hi), adr(inst.x_lo), adr(inst.x_hi))


class Problem:
    """A batch of robust trajectory problems resident on the GPU."""

    _COUNTS = {
        F_XHAT: lambda x: (x.T + 1) * x.nx, F_DX: lambda x: (x.T + 1) * x.nx, F_UHAT: lambda x: x.T * x.nu,
        F_DU: lambda x: x.T * x.nu, F_A: lambda x: x.T * x.nx * x.nx, F_B: lambda x: x.T * x.nx * x.nu,
        F_G0: lambda x: x.n_rows, F_P: lambda x: x.n_rows, F_PT: lambda x: x.n_rows, F_LAMP: lambda x: x.n_rows,
        F_BHAT: lambda x: x.n_entries_state, F_BVEC: lambda x: x.n_entries_state // x.nx * x.nu,
        F_LAMNU: lambda x: x.n_entries, F_K: lambda x: x.T * x.nu * x.nx, F_KACC: lambda x: x.T * x.nu * x.nx,
        F_GM: lambda x: x.T * x.nu * x.nu, F_SCAL: lambda x: 8, F_STATS: lambda x: 7,
        F_LAMW: lambda x: x.n_rows, F_S: lambda x: x.n_rows, F_LAME: lambda x: (x.T + 1) * x.nx,
    }

    def __init__(self, instances, precision=PREC_FP64, stream=None):
        lib = load()
        self.instances = list(instances)
        self.n = len(self.instances)
        keep = []
        descs = (ProblemDesc * self.n)(*[_desc(x, keep) for x in self.instances])
        h = C.c_void_p()
        _check(lib.nrto_problem_create(descs, self.n, precision, C.c_void_p(stream), C.byref(h)))
        self._h = h
        self.precision = precision
        self.info = []
        for i in range(self.n):
            inf = InstanceInfo()
            _check(lib.nrto_problem_info(h, i, C.byref(inf)))
            self.info.append(inf)

    def close(self):
        if getattr(self, "_h", None):
            load().nrto_problem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_rows(self, i=None):
        return self.info[i].n_rows if i is not None else sum(x.n_rows for x in self.info)

    def _cat(self, per):
        return int(sum(per(x) for x in self.info))

    def _split(self, flat, shape):
        out, o = [], 0
        for x in self.info:
            s = shape(x)
            n = int(np.prod(s))
            out.append(flat[o:o + n].reshape(s))
            o += n
        return out

    def update(self, instances):
        keep = []
        descs = (ProblemDesc * self.n)(*[_desc(x, keep) for x in instances])
        _check(load().nrto_problem_update(self._h, descs, self.n))

    def linearize(self, u_hat=None):
        u = None if u_hat is None else np.ascontiguousarray(np.concatenate([np.asarray(x).reshape(-1) for x in u_hat]))
        _check(load().nrto_linearize(self._h, _ptr(u)))

    def set_trust_radius(self, r):
        r = np.ascontiguousarray(np.broadcast_to(np.asarray(r, dtype=np.float64), (self.n,)).copy())
        _check(load().nrto_set_trust_radius(self._h, _ptr(r)))

    def solve_socp(self, opts: Options, fetch=True):
        o = opts.c()
        if not fetch:
            return _check(load().nrto_solve_socp(self._h, C.byref(o), None), allow=(3,))
        du = np.zeros(self._cat(lambda x: x.T * x.nu))
        K = np.zeros(self._cat(lambda x: x.T * x.nu * x.nx))
        p = np.zeros(self.n_rows())
        pt = np.zeros(self.n_rows())
        it = np.zeros(self.n, dtype=np.int32)
        rp = np.zeros(self.n)
        rd = np.zeros(self.n)
        st = np.zeros(self.n, dtype=np.int32)
        out = SocpOut(_ptr(du), _ptr(K), _ptr(p), _ptr(pt), it.ctypes.data_as(_ip), _ptr(rp), _ptr(rd),
                      st.ctypes.data_as(_ip))
        code = _check(load().nrto_solve_socp(self._h, C.byref(o), C.byref(out)), allow=(3,))
        return dict(du=self._split(du, lambda x: (x.T, x.nu)), K=self._split(K, lambda x: (x.T, x.nu, x.nx)),
                    p=self._split(p, lambda x: (x.n_rows,)), pt=self._split(pt, lambda x: (x.n_rows,)),
                    iters=it, r_p=rp, r_d=rd, status=st, code=code)

    def outer_step(self, opts: Options):
        acc = np.zeros(self.n, dtype=np.int32)
        _check(load().nrto_outer_step(self._h, C.byref(opts.c()), acc.ctypes.data_as(_ip)))
        return acc

    def solve(self, opts: Options, n_outer=10, fetch=True):
        o = opts.c()
        if not fetch:
            return _check(load().nrto_solve(self._h, C.byref(o), n_outer, None, None, None))
        u = np.zeros(self._cat(lambda x: x.T * x.nu))
        K = np.zeros(self._cat(lambda x: x.T * x.nu * x.nx))
        m = np.zeros(self.n)
        _check(load().nrto_solve(self._h, C.byref(o), n_outer, _ptr(u), _ptr(K), _ptr(m)))
        return dict(u_bar=self._split(u, lambda x: (x.T, x.nu)), K=self._split(K, lambda x: (x.T, x.nu, x.nx)),
                    merit=m)

    def set_warm_start(self, K, pt, lam_p):
        K = np.ascontiguousarray(np.concatenate([np.asarray(k).reshape(-1) for k in K]))
        pt = np.ascontiguousarray(np.concatenate([np.asarray(k).reshape(-1) for k in pt]))
        lp = np.ascontiguousarray(np.concatenate([np.asarray(k).reshape(-1) for k in lam_p]))
        _check(load().nrto_set_warm_start(self._h, _ptr(K), _ptr(pt), _ptr(lp)))

    def set_warm_start_lifted(self, theta, lam_w, du, lam_e, rho=None):
        """The lifted warm start (nrto_set_warm_start_lifted) after set_warm_start: per instance θ and
        λ_w per row, δû (T, nu), λ_e (T, nx) for steps 1..T, and optionally the penalty per instance."""
        cat = lambda a: np.ascontiguousarray(np.concatenate([np.asarray(k, dtype=np.float64).reshape(-1) for k in a]))
        r = None if rho is None else np.ascontiguousarray(np.broadcast_to(np.asarray(rho, dtype=np.float64), (self.n,)).copy())
        _check(load().nrto_set_warm_start_lifted(self._h, _ptr(cat(theta)), _ptr(cat(lam_w)), _ptr(cat(du)),
                                                 _ptr(cat(lam_e)), _ptr(r)))

    def set_warm_start_from_network_lifted(self, net, features, row_map, offsets):
        """Network forward on the device and scatter into the lifted warm start; offsets of K, p̃, λ_p,
        θ, λ_w, δû, λ_e and log ρ (-1: the solver's ρ) in the network output."""
        f = np.ascontiguousarray(np.asarray(features, dtype=np.float32))
        m = np.ascontiguousarray(np.asarray(row_map, dtype=np.int32))
        o = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
        assert f.shape[0] == self.n and m.size == self.n_rows() and o.size == 8
        _check(load().nrto_set_warm_start_from_network_lifted(self._h, net._h, f.ctypes.data_as(C.POINTER(C.c_float)),
                                                              m.ctypes.data_as(_ip), o.ctypes.data_as(_ip)))

    def set_warm_start_from_network(self, net, features, row_map, k_off, pt_off, lp_off):
        """Network forward on the device and scatter into the next inner solve's (K, p̃, λ_p)."""
        f = np.ascontiguousarray(np.asarray(features, dtype=np.float32))
        m = np.ascontiguousarray(np.asarray(row_map, dtype=np.int32))
        assert f.shape[0] == self.n and m.size == self.n_rows()
        _check(load().nrto_set_warm_start_from_network(self._h, net._h, f.ctypes.data_as(C.POINTER(C.c_float)),
                                                       m.ctypes.data_as(_ip), int(k_off), int(pt_off), int(lp_off)))

    def export(self, field, i):
        n = int(self._COUNTS[field](self.info[i]))
        out = np.zeros(n)
        _check(load().nrto_export(self._h, field, i, _ptr(out), n))
        return out

    def import_(self, field, i, values):
        v = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(-1))
        _check(load().nrto_import(self._h, field, i, _ptr(v), v.size))

    def profile(self, enable=True):
        """(solver-kernel ms, launches) since the previous call; then enable/disable recording."""
        ms = C.c_double()
        n = C.c_longlong()
        _check(load().nrto_profile(self._h, int(enable), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    PHASES = ["init", "rows", "control+reduce", "slacks", "riccati_terms", "gain_solve", "riccati_sweep", "duals",
              "rows_copy_wait"]

    def phase_cycles(self):
        """Per-phase SM cycles (summed over CTAs) recorded while profiling was enabled; clears them."""
        buf = (C.c_longlong * 9)()
        _check(load().nrto_phase_cycles(self._h, buf, 9))
        return dict(zip(self.PHASES, [int(x) for x in buf]))

    def kernel_launches(self):
        return int(load().nrto_kernel_launches(self._h))

    def set_graph(self, enable=True):
        """Capture / replay nrto_solve's launch sequence as a CUDA graph (default on)."""
        _check(load().nrto_set_graph(self._h, int(enable)))

    def set_launch_mapping(self, mapping):
        _check(load().nrto_set_launch_mapping(self._h, int(mapping)))

    def autotune(self, opts: Options, n_outer=1, reps=1):
        """Time every launch mapping on this batch and keep the fastest: (chosen, ms per mapping)."""
        ms = np.zeros(NMAPPING)
        ch = C.c_int(-1)
        _check(load().nrto_autotune(self._h, C.byref(opts.c()), int(n_outer), int(reps), _ptr(ms), C.byref(ch)))
        return ch.value, ms

    def graph_info(self):
        """(captures, replays) of nrto_solve's CUDA graph."""
        c, r = C.c_longlong(0), C.c_longlong(0)
        _check(load().nrto_graph_info(self._h, C.byref(c), C.byref(r)))
        return c.value, r.value

    STATS = ["cum_iters", "iters", "status", "n_accepted", "rho", "dr_iters", "fallback", "accepted_status",
             "merit", "cost", "max_violation", "trust_radius", "r_p", "r_d", "pcg_iters"]

    def stats(self):
        """Per-instance statistics of the batch (nrto_get_stats): a dict of arrays named by STATS."""
        out = np.zeros((self.n, NSTAT))
        _check(load().nrto_get_stats(self._h, _ptr(out), NSTAT))
        return {k: out[:, i] for i, k in enumerate(self.STATS)}

    def monte_carlo(self, n_interior=1000, n_edge=1000, seed=0, tol=0.0, K=None, per_sample=False):
        """Monte Carlo robust-constraint satisfaction per instance (nrto_monte_carlo) at the nominal of
        the current linearization, with the gains K (list of (T, nu, nx) arrays, one per instance) or
        those of the accepted iterate.  Returns the satisfied-rollout counts, and with per_sample the
        (n, n_interior + n_edge) worst constraint values as well."""
        ok = np.zeros(self.n, dtype=np.int32)
        Kf = None
        if K is not None:
            Kf = np.ascontiguousarray(np.concatenate([np.asarray(k, dtype=np.float64).reshape(-1) for k in K]))
        worst = np.zeros((self.n, n_interior + n_edge)) if per_sample else None
        _check(load().nrto_monte_carlo(self._h, _ptr(Kf), n_interior, n_edge, seed, tol,
                                       ok.ctypes.data_as(_ip), _ptr(worst)))
        return (ok, worst) if per_sample else ok


def solve_noalloc(instances, opts: Options, n_outer=10, precision=PREC_FP64, stream=None):
    """Problem(instances).solve(opts, n_outer) without any device allocation: the batch lives in the
    library's static device area (for callers that cannot allocate device memory).  Returns the same
    dict as Problem.solve."""
    insts = list(instances)
    keep = []
    descs = (ProblemDesc * len(insts))(*[_desc(x, keep) for x in insts])
    u = np.zeros(sum(x.T * x.nu for x in insts))
    K = np.zeros(sum(x.T * x.nu * x.nx for x in insts))
    m = np.zeros(len(insts))
    o = opts.c()
    _check(load().nrto_solve_noalloc(descs, len(insts), precision, C.byref(o), n_outer, C.c_void_p(stream),
                                     _ptr(u), _ptr(K), _ptr(m)))
    us, Ks, a, b = [], [], 0, 0
    for x in insts:
        us.append(u[a:a + x.T * x.nu].reshape(x.T, x.nu))
        Ks.append(K[b:b + x.T * x.nu * x.nx].reshape(x.T, x.nu, x.nx))
        a += x.T * x.nu
        b += x.T * x.nu * x.nx
    return dict(u_bar=us, K=Ks, merit=m)


def selftest_bounded_wait(stream=None):
    """Run the solver kernels' bounded copy wait against a barrier that never completes
    (nrto_selftest_bounded_wait): (status, SM cycles waited); status 4 means the wait gave up."""
    st = C.c_int(0)
    cyc = C.c_longlong(0)
    _check(load().nrto_selftest_bounded_wait(C.c_void_p(stream), C.byref(st), C.byref(cyc)))
    return st.value, cyc.value


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


class MLP:
    """The warm-start network on the GPU (nrto_mlp_*): GELU hidden layers, masked MSE, Adam.
    Parameters travel as one flat float32 array: per layer W (out, in) row-major, then b."""

    def __init__(self, dims, max_batch, stream=None):
        lib = load()
        self.dims = [int(d) for d in dims]
        self.max_batch = int(max_batch)
        arr = (C.c_int * len(self.dims))(*self.dims)
        h = C.c_void_p()
        _check(lib.nrto_mlp_create(arr, len(self.dims), self.max_batch, C.c_void_p(stream), C.byref(h)))
        self._h = h
        self.n_params = int(lib.nrto_mlp_num_params(h))

    def close(self):
        if getattr(self, "_h", None):
            load().nrto_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pack(self, W, b):
        return np.concatenate([np.concatenate([w.reshape(-1), bb.reshape(-1)]) for w, bb in zip(W, b)]).astype(np.float32)

    def unpack(self, flat):
        W, b, o = [], [], 0
        for din, dout in zip(self.dims[:-1], self.dims[1:]):
            W.append(flat[o:o + din * dout].reshape(dout, din))
            o += din * dout
            b.append(flat[o:o + dout].copy())
            o += dout
        return W, b

    def set_params(self, flat):
        f = _f32(flat)
        assert f.size == self.n_params
        _check(load().nrto_mlp_set_params(self._h, f.ctypes.data_as(C.POINTER(C.c_float))))

    def get_params(self):
        f = np.zeros(self.n_params, dtype=np.float32)
        _check(load().nrto_mlp_get_params(self._h, f.ctypes.data_as(C.POINTER(C.c_float))))
        return f

    def forward(self, x):
        x = _f32(x)
        y = np.zeros((x.shape[0], self.dims[-1]), dtype=np.float32)
        _fp = C.POINTER(C.c_float)
        _check(load().nrto_mlp_forward(self._h, x.ctypes.data_as(_fp), x.shape[0], y.ctypes.data_as(_fp)))
        return y

    def train_step(self, x, t, mask, lr, want_grads=False):
        x, t, mask = _f32(x), _f32(t), _f32(mask)
        _fp = C.POINTER(C.c_float)
        loss = C.c_double(0.0)
        g = np.zeros(self.n_params, dtype=np.float32) if want_grads else None
        _check(load().nrto_mlp_train_step(self._h, x.ctypes.data_as(_fp), t.ctypes.data_as(_fp),
                                          mask.ctypes.data_as(_fp), x.shape[0], float(lr), C.byref(loss),
                                          g.ctypes.data_as(_fp) if g is not None else None))
        return (loss.value, g) if want_grads else loss.value

    def kernel_launches(self):
        return int(load().nrto_mlp_kernel_launches(self._h))

    def profile(self, enable=True):
        """(GEMM ms, GEMM FLOPs, GEMM launches) since the previous call; then enable/disable timing."""
        ms, fl, n = C.c_double(0), C.c_double(0), C.c_longlong(0)
        _check(load().nrto_mlp_profile(self._h, int(enable), C.byref(ms), C.byref(fl), C.byref(n)))
        return ms.value, fl.value, n.value
