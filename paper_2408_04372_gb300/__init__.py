"""Python binding of libstmg (include/stmg.h): argument marshalling only.

Every step of the space-time multigrid path runs in the CUDA library; this
module converts torch tensors to device pointers and checks sizes.  There is no
CPU fallback: importing works without a GPU, but creating a context needs the
compiled library and a CUDA device and fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os
import weakref

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstmg.so")

HEAT, WAVE = 0, 1
DG, CGP = 0, 1
COEFF_PER_CELL, COEFF_PER_QPOINT = 0, 1
FP64, FP32, BF16, DF32, FP8 = 1, 2, 3, 4, 5
SMOOTHER_AUTO, SMOOTHER_DENSE, SMOOTHER_FD, SMOOTHER_EIG, SMOOTHER_EIG_TC = 0, 1, 2, 3, 4
COARSEN_P_THEN_H, COARSEN_H = 0, 1

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NOT_CONVERGED", 5: "BREAKDOWN",
          6: "TIMEOUT", 7: "NONFINITE", 8: "INTERNAL", 9: "UNSUPPORTED"}

EXPORTS = ["stmg_create", "stmg_destroy", "stmg_last_error", "stmg_sizes", "stmg_level_info",
           "stmg_node_coords", "stmg_qpoint_coords", "stmg_apply", "stmg_residual", "stmg_smooth",
           "stmg_restrict", "stmg_prolongate_add", "stmg_vcycle", "stmg_rhs", "stmg_solve",
           "stmg_wave_velocity", "stmg_guess_previous", "stmg_solve_slab_host", "stmg_launch_count",
           "stmg_time_kernel", "stmg_smooth_noalloc", "stmg_net_create", "stmg_net_destroy", "stmg_net_predict",
           "stmg_net_train_step", "stmg_net_gradients", "stmg_net_weights", "stmg_select_guess",
           "stmg_solve_slab_host_learned", "stmg_selftest_device_timeout", "stmg_level_slabs", "stmg_point_values"]
KERNEL_APPLY, KERNEL_ASM, KERNEL_VCYCLE, KERNEL_ORTHO = 1, 2, 3, 4


class StmgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"stmg {STATUS.get(status, status)}: {msg}")
        self.status = status


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_cells", ctypes.c_int), ("vertices", ctypes.POINTER(ctypes.c_double))]


class Problem(ctypes.Structure):
    _fields_ = [("pde", ctypes.c_int), ("time_scheme", ctypes.c_int), ("p", ctypes.c_int), ("k", ctypes.c_int),
                ("tau", ctypes.c_double), ("coeff_mode", ctypes.c_int), ("coeff", ctypes.POINTER(ctypes.c_double)),
                ("n_slabs", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("vcycle_precision", ctypes.c_int),
                ("inverse_precision", ctypes.c_int), ("smoother_kind", ctypes.c_int),
                ("omega", ctypes.POINTER(ctypes.c_double)), ("fgmres_restart", ctypes.c_int),
                ("rtol", ctypes.c_double), ("max_it", ctypes.c_int), ("outer_apply", ctypes.c_int),
                ("atol", ctypes.c_double), ("space_coarsening", ctypes.c_int), ("coarse_max_dofs", ctypes.c_int),
                ("asm_weighting", ctypes.c_int), ("outer_relax", ctypes.c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("initial_rel_residual", ctypes.c_double), ("relaxed_iterations", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libstmg.so (build it with paper_2408_04372_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_2408_04372_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    sig = {
        "stmg_create": [ctypes.POINTER(vp), ctypes.POINTER(Mesh), ctypes.POINTER(Problem), ctypes.POINTER(Options), vp],
        "stmg_destroy": [vp],
        "stmg_sizes": [vp, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "stmg_level_info": [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                            ctypes.POINTER(i64), ctypes.POINTER(i32), dp],
        "stmg_level_slabs": [vp, i32, ctypes.POINTER(i32), dp],
        "stmg_point_values": [vp, vp, i32, vp, vp],
        "stmg_node_coords": [vp, i32, vp],
        "stmg_qpoint_coords": [vp, i32, vp],
        "stmg_apply": [vp, i32, i32, vp, vp],
        "stmg_residual": [vp, i32, i32, vp, vp, vp],
        "stmg_smooth": [vp, i32, i32, i32, vp, vp],
        "stmg_restrict": [vp, i32, i32, vp, vp],
        "stmg_prolongate_add": [vp, i32, i32, vp, vp],
        "stmg_vcycle": [vp, i32, vp, vp],
        "stmg_rhs": [vp, vp, vp, vp, vp, vp],
        "stmg_solve": [vp, vp, vp, ctypes.POINTER(SolveStats)],
        "stmg_wave_velocity": [vp, vp, vp, vp, vp],
        "stmg_guess_previous": [vp, vp, vp],
        "stmg_solve_slab_host": [vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(SolveStats)],
        "stmg_launch_count": [vp, ctypes.POINTER(i64)],
        "stmg_selftest_device_timeout": [vp],
        "stmg_smooth_noalloc": [vp, i32, i32, i32, vp, vp],
        "stmg_net_create": [ctypes.POINTER(vp), vp, i32, ctypes.POINTER(i32), dp, dp, dp],
        "stmg_net_destroy": [vp],
        "stmg_net_predict": [vp, vp, vp, vp],
        "stmg_net_train_step": [vp, vp, vp, vp, ctypes.c_double, dp],
        "stmg_net_gradients": [vp, vp, vp, vp, dp, dp, dp, dp],
        "stmg_net_weights": [vp, dp, dp],
        "stmg_select_guess": [vp, vp, vp, vp, ctypes.POINTER(i32)],
        "stmg_solve_slab_host_learned": [vp, vp, vp, vp, vp, ctypes.POINTER(i32), ctypes.POINTER(SolveStats)],
        "stmg_time_kernel": [vp, i32, i32, i32, i32, dp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.stmg_last_error.argtypes = [vp]
    lib.stmg_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _dptr(a):
    """Host numpy float64 array -> double* (None -> NULL)."""
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Context:
    """One STMG hierarchy on the current CUDA device and stream."""

    def __init__(self, dim, n_cells, p, k, tau, pde=HEAT, scheme=DG, vertices=None, coeff=None,
                 coeff_mode=COEFF_PER_CELL, nu_pre=1, nu_post=1, vcycle_precision=FP32, inverse_precision=0,
                 omega=None, restart=30, rtol=1e-8, max_it=200, stream=None, smoother_kind=SMOOTHER_AUTO,
                 outer_apply=0, atol=0.0, space_coarsening=0, coarse_max_dofs=0, n_slabs=1, asm_weighting=0,
                 outer_relax=0):
        import numpy as np
        import torch
        self.lib = load()
        self._keep = []
        self._nets = weakref.WeakSet()
        v = None if vertices is None else np.ascontiguousarray(vertices, dtype=np.float64)
        c = None if coeff is None else np.ascontiguousarray(coeff, dtype=np.float64)
        om = None if omega is None else np.ascontiguousarray(omega, dtype=np.float64)
        self._keep += [v, c, om]
        mesh = Mesh(dim, n_cells, _dptr(v))
        prob = Problem(pde, scheme, p, k, float(tau), coeff_mode, _dptr(c), int(n_slabs))
        opts = Options(nu_pre, nu_post, vcycle_precision, inverse_precision, smoother_kind, _dptr(om), restart, rtol,
                       max_it, outer_apply, float(atol), space_coarsening, coarse_max_dofs, asm_weighting, outer_relax)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = self.lib.stmg_create(ctypes.byref(h), ctypes.byref(mesh), ctypes.byref(prob), ctypes.byref(opts),
                                  ctypes.c_void_p(stream.cuda_stream))
        self.h = h
        if st != 0:
            msg = self.lib.stmg_last_error(h).decode()
            self.lib.stmg_destroy(h)
            self.h = None
            raise StmgError(st, msg)
        n_nodes, nt, nl = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.stmg_sizes(h, ctypes.byref(n_nodes), ctypes.byref(nt), ctypes.byref(nl)))
        self.n_nodes, self.nt, self.n_levels, self.dim = n_nodes.value, nt.value, nl.value, dim
        self.pde = pde
        self.n_slabs = int(n_slabs)
        self.size = self.n_slabs * self.nt * self.n_nodes  # finest-level vector length, [slab][N_t][node]

    def __del__(self):
        for net in list(getattr(self, "_nets", ())):
            net.close()
        if getattr(self, "h", None):
            self.lib.stmg_destroy(self.h)
            self.h = None

    def close(self):
        self.__del__()

    def _check(self, st):
        if st != 0:
            raise StmgError(st, self.lib.stmg_last_error(self.h).decode())

    def level_info(self, level):
        p, N, k, nt = (ctypes.c_int() for _ in range(4))
        nn, om = ctypes.c_int64(), ctypes.c_double()
        self._check(self.lib.stmg_level_info(self.h, level, ctypes.byref(p), ctypes.byref(N), ctypes.byref(k),
                                             ctypes.byref(nn), ctypes.byref(nt), ctypes.byref(om)))
        nc, tau = ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.stmg_level_slabs(self.h, level, ctypes.byref(nc), ctypes.byref(tau)))
        return dict(p=p.value, n_cells=N.value, k=k.value, n_nodes=nn.value, nt=nt.value, omega=om.value,
                    n_slabs=nc.value, tau=tau.value)

    def point_values(self, u, points):
        """u (float64 CUDA tensor, n_slabs * N_t * n_nodes) at physical points (npts x dim) ->
        numpy (npts, n_slabs * N_t): every slab's time DoFs (goal quantities)."""
        import numpy as np
        import torch
        self._vec(u)
        if u.dtype != torch.float64:
            raise TypeError("point_values takes a float64 vector")
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, self.dim)
        out = np.zeros((len(pts), self.n_slabs * self.nt))
        self._check(self.lib.stmg_point_values(self.h, _ptr(u), len(pts), pts.ctypes.data_as(ctypes.c_void_p),
                                               out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def node_coords(self, level=0):
        import numpy as np
        info = self.level_info(level)
        out = np.zeros((info["n_nodes"], self.dim))
        self._check(self.lib.stmg_node_coords(self.h, level, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def qpoint_coords(self, level=0):
        import numpy as np
        info = self.level_info(level)
        nq = (info["p"] + 1) ** self.dim
        out = np.zeros((info["n_cells"] ** self.dim, nq, self.dim))
        self._check(self.lib.stmg_qpoint_coords(self.h, level, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    @staticmethod
    def _prec(t):
        import torch
        if t.dtype == torch.float64:
            return FP64
        if t.dtype == torch.float32:
            return FP32
        raise TypeError("vectors must be float32 or float64")

    @staticmethod
    def _same(*ts):
        """The library reads every vector of one call in the precision of the last one: all must agree."""
        ts = [t for t in ts if t is not None]
        if any(t.dtype != ts[0].dtype or t.device != ts[0].device for t in ts):
            raise TypeError("vectors of one call must share dtype and device")

    def _vec(self, t, level=0):
        if t is None:
            return
        info = self.level_info(level)
        if not t.is_cuda or not t.is_contiguous() or t.numel() != info["n_slabs"] * info["nt"] * info["n_nodes"]:
            raise ValueError("expected a contiguous CUDA tensor of n_slabs * N_t * n_nodes values")

    def apply(self, x, y, level=0):
        self._vec(x, level); self._vec(y, level)
        self._same(x, y)
        self._check(self.lib.stmg_apply(self.h, level, self._prec(x), _ptr(x), _ptr(y)))

    def apply_df(self, x, y):
        """y (FP64) = S x (FP32) on level 0 in double-float arithmetic (outer_apply = DF32)."""
        import torch
        self._vec(x, 0); self._vec(y, 0)
        if x.dtype != torch.float32 or y.dtype != torch.float64:
            raise TypeError("apply_df takes a float32 x and a float64 y")
        self._check(self.lib.stmg_apply(self.h, 0, DF32, _ptr(x), _ptr(y)))

    def residual(self, f, u, r, level=0):
        for t in (f, u, r):
            self._vec(t, level)
        self._same(f, u, r)
        self._check(self.lib.stmg_residual(self.h, level, self._prec(u), _ptr(f), _ptr(u), _ptr(r)))

    def smooth(self, f, u, sweeps=1, level=0):
        self._vec(f, level); self._vec(u, level)
        self._same(f, u)
        self._check(self.lib.stmg_smooth(self.h, level, self._prec(u), sweeps, _ptr(f), _ptr(u)))

    def smooth_noalloc(self, f, u, sweeps=1, level=0):
        """stmg_smooth without device allocation: residual scratch in the library's fixed buffer."""
        self._vec(f, level); self._vec(u, level)
        self._same(f, u)
        self._check(self.lib.stmg_smooth_noalloc(self.h, level, self._prec(u), sweeps, _ptr(f), _ptr(u)))

    def restrict(self, r_fine, r_coarse, level=0):
        self._vec(r_fine, level); self._vec(r_coarse, level + 1)
        self._same(r_fine, r_coarse)
        self._check(self.lib.stmg_restrict(self.h, level, self._prec(r_fine), _ptr(r_fine), _ptr(r_coarse)))

    def prolongate_add(self, e_coarse, u_fine, level=0):
        self._vec(e_coarse, level + 1); self._vec(u_fine, level)
        self._same(e_coarse, u_fine)
        self._check(self.lib.stmg_prolongate_add(self.h, level, self._prec(u_fine), _ptr(e_coarse), _ptr(u_fine)))

    def vcycle(self, r, e):
        self._vec(r); self._vec(e)
        self._same(r, e)
        self._check(self.lib.stmg_vcycle(self.h, self._prec(r), _ptr(r), _ptr(e)))

    def rhs(self, f, rhs, f0=None, u0=None, v0=None):
        self._check(self.lib.stmg_rhs(self.h, _ptr(f), _ptr(f0), _ptr(u0), _ptr(v0), _ptr(rhs)))

    def solve(self, rhs, u):
        st = SolveStats()
        code = self.lib.stmg_solve(self.h, _ptr(rhs), _ptr(u), ctypes.byref(st))
        if code not in (0, 4):
            self._check(code)
        return dict(iterations=st.iterations, restarts=st.restarts, rel_residual=st.rel_residual,
                    initial_rel_residual=st.initial_rel_residual, relaxed_iterations=st.relaxed_iterations,
                    converged=code == 0)

    def wave_velocity(self, u, u0, v0, v):
        self._check(self.lib.stmg_wave_velocity(self.h, _ptr(u), _ptr(u0), _ptr(v0), _ptr(v)))

    def select_guess(self, rhs, candidate, u):
        """u = candidate if it has the smaller FP64 residual; returns True when taken."""
        c = ctypes.c_int()
        self._check(self.lib.stmg_select_guess(self.h, _ptr(rhs), _ptr(candidate), _ptr(u), ctypes.byref(c)))
        return bool(c.value)

    def guess_previous(self, u0, u):
        self._check(self.lib.stmg_guess_previous(self.h, _ptr(u0), _ptr(u)))

    def launch_count(self):
        c = ctypes.c_int64()
        self._check(self.lib.stmg_launch_count(self.h, ctypes.byref(c)))
        return c.value

    def selftest_device_timeout(self):
        """Runs the bounded-wait test hook; returns the status code (STMG_ERR_TIMEOUT = 6 expected)."""
        return self.lib.stmg_selftest_device_timeout(self.h)

    def time_kernel(self, kernel, level=0, precision=FP64, reps=20):
        """Mean duration in ms of one kernel, CUDA events on the context's own stream."""
        ms = ctypes.c_double()
        self._check(self.lib.stmg_time_kernel(self.h, kernel, level, precision, reps, ctypes.byref(ms)))
        return ms.value

    def solve_slab_host(self, f, u0, f0=None, v0=None, want_v=False, out_u=None):
        """Host numpy in/out: f (N_t, n) source at the slab's time nodes, u0 (n,) previous end value."""
        import numpy as np
        f = np.ascontiguousarray(f, dtype=np.float64)
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        f0 = None if f0 is None else np.ascontiguousarray(f0, dtype=np.float64)
        v0 = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
        u = np.zeros((self.nt, self.n_nodes)) if out_u is None else out_u
        v = np.zeros((self.nt, self.n_nodes)) if want_v else None
        st = SolveStats()
        vp = lambda a: ctypes.c_void_p(0) if a is None else a.ctypes.data_as(ctypes.c_void_p)
        code = self.lib.stmg_solve_slab_host(self.h, vp(f), vp(f0), vp(u0), vp(v0), vp(u), vp(v), ctypes.byref(st))
        if code not in (0, 4):
            self._check(code)
        stats = dict(iterations=st.iterations, rel_residual=st.rel_residual, converged=code == 0)
        return (u, v, stats) if want_v else (u, stats)


class Net:
    """Learned initial guess bound to a context (stmg_net_* in include/stmg.h)."""

    def __init__(self, ctx: Context, channels, weights, biases, scales):
        import numpy as np
        self.ctx, self.lib = ctx, ctx.lib
        self.channels = list(channels)
        self.L = len(channels) - 1
        w = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(-1) for x in weights]))
        b = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(-1) for x in biases]))
        sc = np.ascontiguousarray(np.asarray(scales, np.float64))
        ch = (ctypes.c_int * len(channels))(*channels)
        h = ctypes.c_void_p()
        ctx._check(self.lib.stmg_net_create(ctypes.byref(h), ctx.h, self.L, ch, _dptr(w), _dptr(b), _dptr(sc)))
        self.h = h
        ctx._nets.add(self)
        self._nw, self._nb = w.size, b.size

    def close(self):
        if getattr(self, "h", None):
            self.lib.stmg_net_destroy(self.h)
            self.h = None

    __del__ = close

    def _split(self, flat_w, flat_b):
        W, B, ow, ob = [], [], 0, 0
        for l in range(self.L):
            ci, co = self.channels[l], self.channels[l + 1]
            W.append(flat_w[ow:ow + co * ci * 27].reshape(co, ci, 27))
            B.append(flat_b[ob:ob + co])
            ow += co * ci * 27
            ob += co
        return W, B

    def predict(self, u_prev, f, guess):
        self.ctx._check(self.lib.stmg_net_predict(self.h, _ptr(u_prev), _ptr(f), _ptr(guess)))

    def train_step(self, u_prev, f, u_target, lr):
        loss = ctypes.c_double()
        self.ctx._check(self.lib.stmg_net_train_step(self.h, _ptr(u_prev), _ptr(f), _ptr(u_target), lr,
                                                     ctypes.byref(loss)))
        return loss.value

    def gradients(self, u_prev, f, u_target):
        import numpy as np
        gw, gb = np.zeros(self._nw), np.zeros(self._nb)
        out = np.zeros((self.ctx.nt, self.ctx.n_nodes))
        loss = ctypes.c_double()
        self.ctx._check(self.lib.stmg_net_gradients(self.h, _ptr(u_prev), _ptr(f), _ptr(u_target), ctypes.byref(loss),
                                                    _dptr(gw), _dptr(gb), _dptr(out)))
        W, B = self._split(gw, gb)
        return loss.value, W, B, out

    def solve_slab_host(self, f, u_prev, out_u):
        """Host numpy in/out learned slab step; returns (stats dict, network guess taken)."""
        import numpy as np
        f = np.ascontiguousarray(f, dtype=np.float64)
        u_prev = np.ascontiguousarray(u_prev, dtype=np.float64)
        st, ch = SolveStats(), ctypes.c_int()
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        code = self.lib.stmg_solve_slab_host_learned(self.ctx.h, self.h, vp(f), vp(u_prev), vp(out_u),
                                                     ctypes.byref(ch), ctypes.byref(st))
        if code not in (0, 4):
            self.ctx._check(code)
        return dict(iterations=st.iterations, rel_residual=st.rel_residual, converged=code == 0), bool(ch.value)

    def weights(self):
        import numpy as np
        w, b = np.zeros(self._nw), np.zeros(self._nb)
        self.ctx._check(self.lib.stmg_net_weights(self.h, _dptr(w), _dptr(b)))
        return self._split(w, b)
