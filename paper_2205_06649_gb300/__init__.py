"""GB300-native space-time domain-decomposed 4D-Var (DD-4DVar) hot path.

Python binding of the C ABI in include/dd4dvar.h: one ``Context`` object
wraps one ``dd4dv_ctx``; its methods carry the C names without the
``dd4dv_`` prefix and only marshal arguments (numpy arrays -> host pointers,
CUDA torch tensors -> device pointers).  Every step of the computation runs in
the library's CUDA kernels; there is no CPU fallback.

Method: D'Amore, Constantinescu & Carracciuolo, arXiv 2205.06649 (Alg. 1,
local functional Eq. eq:cost:parallel1, shallow-water model of Sec. 7).
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import _abi

__all__ = ["Context", "DD4DVError", "lib", "solver_defaults"]

lib = _abi.load()

# dd4dv_sweep_kernels codes
KERNEL_NAMES = {1: "stripe", 2: "deep-halo", 3: "stripe-4buf", 4: "stripe-2buf"}


class DD4DVError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_abi.STATUS.get(status, status)}: {msg}")
        self.status = status


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _ptr(x, dtype, device: bool):
    """Data pointer of a contiguous array of the given dtype (numpy for host,
    torch CUDA tensor for device)."""
    if x is None:
        return None
    if device:
        if not _is_torch_cuda(x):
            raise TypeError("device call needs CUDA torch tensors")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        want = {np.float64: "torch.float64", np.int32: "torch.int32"}[dtype]
        if str(x.dtype) != want:
            raise TypeError(f"expected {want}, got {x.dtype}")
        return C.c_void_p(x.data_ptr())
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
    return C.c_void_p(x.ctypes.data)


def solver_defaults(**kw) -> _abi.dd4dv_solver:
    s = _abi.dd4dv_solver(lbfgs_m=5, max_local_iters=20, max_trials=20, max_outer=10,
                          eps_outer=1e-6, gtol_rel=1e-6, c1=1e-4, use_graphs=1, local_solver=0,
                          gn_iters=3, cg_iters=10, cg_tol=1e-6)
    for k, v in kw.items():
        setattr(s, k, v)
    return s


class Context:
    """One DD-4DVar problem on the current CUDA device (dd4dv_ctx)."""

    def __init__(self, nlon: int, nlat: int, dt: float, nsteps: int, precision: int = 0,
                 lat_min_deg: float = -80.0, lat_max_deg: float = 80.0, radius: float = 6.371e6,
                 gravity: float = 9.81, omega: float = 7.292e-5, h_ref: float = 4000.0,
                 stream: Optional[int] = None):
        """stream: handle of a CUDA stream for the library's work; by default a
        new torch stream.  Calls with CUDA tensors are ordered after the work
        already queued on torch's current stream, and torch's current stream
        waits for them, so tensors can be passed and used like any torch op's."""
        self._tstream = None
        try:
            import torch
            if torch.cuda.is_available():
                self._tstream = (torch.cuda.Stream() if not stream
                                 else torch.cuda.ExternalStream(stream))
                stream = self._tstream.cuda_stream
        except ImportError:
            pass
        self.model = _abi.dd4dv_model(nlon, nlat, lat_min_deg, lat_max_deg, radius, gravity, omega,
                                      dt, nsteps, precision, h_ref)
        h = C.c_void_p()
        st = lib.dd4dv_create(C.byref(self.model), C.c_void_p(stream) if stream else None, C.byref(h))
        if st != 0:
            raise DD4DVError(st, lib.dd4dv_last_error(None).decode())
        self._h = h
        # handle of the stream the library orders its work on (None: its own)
        self.stream = stream if stream else None
        self.nlon, self.nlat, self.nsteps = nlon, nlat, nsteps
        self.n_sub = 0
        self.ctrl_total = 0
        self.traj_total = 0
        self.offsets = np.zeros(1, dtype=np.int64)
        self.traj_offsets = np.zeros(1, dtype=np.int64)
        self.boxes = np.zeros((0, 6), dtype=np.int32)
        self._fwd_token = 0

    def _device_call(self, fn, *tensors):
        """Run a device-pointer call in stream order with torch's current stream."""
        import torch
        cur = torch.cuda.current_stream()
        if self._tstream is not None and self._tstream.cuda_stream != cur.cuda_stream:
            self._tstream.wait_stream(cur)
            st = fn()
            for t in tensors:
                if t is not None:
                    t.record_stream(self._tstream)
            cur.wait_stream(self._tstream)
            return st
        return fn()

    # ---- lifetime ----
    def destroy(self):
        if getattr(self, "_h", None):
            lib.dd4dv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def _check(self, st: int, allow_notconv: bool = False) -> int:
        if st < 0 or (st > 0 and not allow_notconv):
            raise DD4DVError(st, lib.dd4dv_last_error(self._h).decode())
        return st

    def last_error(self) -> str:
        return lib.dd4dv_last_error(self._h).decode()

    # ---- setup (Alg. 1 inputs) ----
    def set_background(self, xb0: np.ndarray):
        xb0 = np.ascontiguousarray(xb0, dtype=np.float64)
        self._check(lib.dd4dv_set_background(self._h, _ptr(xb0, np.float64, False)))

    def set_background_error(self, sigma_b: Sequence[float], corr_len: float = 0.0, rf_passes: int = 4):
        sb = np.ascontiguousarray(sigma_b, dtype=np.float64)
        self._check(lib.dd4dv_set_background_error(self._h, _ptr(sb, np.float64, False), corr_len, rf_passes))

    def set_observations(self, level, var, fi, fj, value, sigma_o):
        lv = np.ascontiguousarray(level, dtype=np.int32)
        vr = np.ascontiguousarray(var, dtype=np.int32)
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (fi, fj, value, sigma_o)]
        self._check(lib.dd4dv_set_observations(self._h, len(lv), _ptr(lv, np.int32, False),
                                               _ptr(vr, np.int32, False),
                                               *[_ptr(x, np.float64, False) for x in a]))

    def set_decomposition(self, P1, P2, Q, o_lon, o_lat, o_t, lon_cuts=None, lat_cuts=None,
                          t_cuts=None, mu=1.0, lam=1.0, weight_obs=1, cluster=0, ckpt_k=0):
        keep = []

        def cuts(c):
            if c is None:
                return None
            arr = np.ascontiguousarray(c, dtype=np.int32)
            keep.append(arr)
            return arr.ctypes.data_as(_abi.c_int_p)
        d = _abi.dd4dv_decomp(P1, P2, Q, cuts(lon_cuts), cuts(lat_cuts), cuts(t_cuts), o_lon, o_lat,
                              o_t, mu, lam, weight_obs, cluster, ckpt_k)
        self._check(lib.dd4dv_set_decomposition(self._h, C.byref(d)))
        n = C.c_int()
        self._check(lib.dd4dv_num_subdomains(self._h, C.byref(n)))
        self.n_sub = n.value
        self.offsets = np.zeros(self.n_sub + 1, dtype=np.int64)
        self.boxes = np.zeros((self.n_sub, 6), dtype=np.int32)
        self._check(lib.dd4dv_control_layout(self._h, C.c_void_p(self.offsets.ctypes.data),
                                             C.c_void_p(self.boxes.ctypes.data)))
        self.traj_offsets = np.zeros(self.n_sub + 1, dtype=np.int64)
        self._check(lib.dd4dv_traj_layout(self._h, C.c_void_p(self.traj_offsets.ctypes.data)))
        self.ctrl_total = int(self.offsets[-1])
        self.traj_total = int(self.traj_offsets[-1])

    # ---- queries ----
    def set_sweep_variant(self, forward: int, adjoint: int = None):
        """Per sweep: 0 = deep-halo FP32 sweep wherever it applies (default),
        1 = stripe sweep only, 2 = the two-buffer stripe forward (x(n) read
        from the stored level) / the four-buffer stripe adjoint (x(n)
        reloaded).  adjoint defaults to the forward's value."""
        adjoint = forward if adjoint is None else adjoint
        self._check(lib.dd4dv_set_sweep_variant(self._h, int(forward), int(adjoint)))

    def sweep_kernels(self) -> dict:
        """Kernels the current shapes run: 1 = stripe sweep, 2 = deep-halo
        sweep, 3 = four-buffer stripe adjoint, 4 = two-buffer stripe
        forward."""
        k = np.zeros(2, dtype=np.int32)
        self._check(lib.dd4dv_sweep_kernels(self._h, C.c_void_p(k.ctypes.data)))
        return {"forward": int(k[0]), "adjoint": int(k[1])}

    def cluster_size(self) -> int:
        """Cluster size of the adjoint sweep."""
        n = C.c_int()
        self._check(lib.dd4dv_cluster_size(self._h, C.byref(n)))
        return n.value

    def sweep_config(self) -> dict:
        sh = np.zeros(5, dtype=np.int32)
        ms = C.c_double()
        self._check(lib.dd4dv_sweep_config(self._h, C.c_void_p(sh.ctypes.data), C.byref(ms)))
        k = C.c_int()
        kms = C.c_double()
        self._check(lib.dd4dv_checkpoint_interval(self._h, C.byref(k), C.byref(kms)))
        kinds = self.sweep_kernels()
        n1 = C.c_int()
        f1 = C.c_double()
        self._check(lib.dd4dv_stage1_stored(self._h, C.byref(n1), C.byref(f1)))
        return {"forward": [int(sh[0]), int(sh[1])], "adjoint": [int(sh[2]), int(sh[3])],
                "stored_stages": bool(sh[4]), "eval_ms": ms.value, "ckpt_k": k.value,
                "x1_stored": {"subdomains": n1.value, "pt_step_share": f1.value},
                "kernels": {"forward": KERNEL_NAMES.get(kinds["forward"], "none"),
                            "adjoint": KERNEL_NAMES.get(kinds["adjoint"], "none")}}

    def set_sweep_config(self, forward, adjoint, stored_stages: bool):
        """forward, adjoint: (cluster size, threads per CTA)."""
        sh = np.array([forward[0], forward[1], adjoint[0], adjoint[1], int(stored_stages)], dtype=np.int32)
        self._check(lib.dd4dv_set_sweep_config(self._h, C.c_void_p(sh.ctypes.data)))

    def pt_steps(self) -> int:
        n = C.c_longlong()
        self._check(lib.dd4dv_pt_steps(self._h, C.byref(n)))
        return n.value

    def launch_count(self) -> int:
        n = C.c_longlong()
        self._check(lib.dd4dv_launch_count(self._h, C.byref(n)))
        return n.value

    def profile_sweeps(self, w, reps: int = 5) -> dict:
        w = np.ascontiguousarray(w, dtype=np.float64)
        ms = np.zeros(4)
        self._check(lib.dd4dv_profile_sweeps(self._h, C.c_void_p(w.ctypes.data), reps,
                                             C.c_void_p(ms.ctypes.data)))
        return dict(forward_ms=ms[0], adjoint_ms=ms[1], eval_ms=ms[2], kernels_per_eval=int(ms[3]))

    # ---- evaluation (host numpy or device torch) ----
    def eval(self, w, grad: bool = True, parts: bool = False):
        self._fwd_token += 1
        dev = _is_torch_cuda(w)
        if dev:
            import torch
            J = torch.empty(self.n_sub, dtype=torch.float64, device=w.device)
            g = torch.empty_like(w) if grad else None
            P = torch.empty(3 * self.n_sub, dtype=torch.float64, device=w.device) if parts else None
        else:
            w = np.ascontiguousarray(w, dtype=np.float64)
            J = np.zeros(self.n_sub)
            g = np.zeros(self.ctrl_total) if grad else None
            P = np.zeros(3 * self.n_sub) if parts else None
        call = lambda: lib.dd4dv_eval(self._h, _ptr(w, np.float64, dev), _ptr(J, np.float64, dev),
                                      _ptr(g, np.float64, dev), _ptr(P, np.float64, dev), int(dev))
        self._check(self._device_call(call, w, J, g, P) if dev else call())
        out = [J]
        if grad:
            out.append(g)
        if parts:
            out.append(P.reshape(self.n_sub, 3))
        return tuple(out) if len(out) > 1 else J

    def forward_token(self) -> int:
        """Counter of dd4dv_eval_forward calls made through this object."""
        return self._fwd_token

    def eval_forward(self, w):
        self._fwd_token += 1
        dev = _is_torch_cuda(w)
        if dev:
            import torch
            J = torch.empty(self.n_sub, dtype=torch.float64, device=w.device)
        else:
            w = np.ascontiguousarray(w, dtype=np.float64)
            J = np.zeros(self.n_sub)
        call = lambda: lib.dd4dv_eval_forward(self._h, _ptr(w, np.float64, dev), _ptr(J, np.float64, dev),
                                              None, int(dev))
        self._check(self._device_call(call, w, J) if dev else call())
        return J

    def eval_backward(self, scale=None, like=None):
        dev = _is_torch_cuda(like) if like is not None else _is_torch_cuda(scale)
        if dev:
            import torch
            g = torch.empty(self.ctrl_total, dtype=torch.float64, device=(like if like is not None else scale).device)
        else:
            g = np.zeros(self.ctrl_total)
            if scale is not None:
                scale = np.ascontiguousarray(scale, dtype=np.float64)
        call = lambda: lib.dd4dv_eval_backward(self._h, _ptr(scale, np.float64, dev), _ptr(g, np.float64, dev),
                                               int(dev))
        self._check(self._device_call(call, scale, g) if dev else call())
        return g

    def tlm(self, w, dw):
        self._fwd_token += 1
        dev = _is_torch_cuda(w)
        if dev:
            import torch
            out = torch.empty(self.traj_total, dtype=torch.float64, device=w.device)
        else:
            w = np.ascontiguousarray(w, dtype=np.float64)
            dw = np.ascontiguousarray(dw, dtype=np.float64)
            out = np.zeros(self.traj_total)
        call = lambda: lib.dd4dv_tlm(self._h, _ptr(w, np.float64, dev), _ptr(dw, np.float64, dev),
                                     _ptr(out, np.float64, dev), int(dev))
        self._check(self._device_call(call, w, dw, out) if dev else call())
        return out

    def adjoint(self, w, y):
        self._fwd_token += 1
        dev = _is_torch_cuda(w)
        if dev:
            import torch
            out = torch.empty(self.ctrl_total, dtype=torch.float64, device=w.device)
        else:
            w = np.ascontiguousarray(w, dtype=np.float64)
            y = np.ascontiguousarray(y, dtype=np.float64)
            out = np.zeros(self.ctrl_total)
        call = lambda: lib.dd4dv_adjoint(self._h, _ptr(w, np.float64, dev), _ptr(y, np.float64, dev),
                                         _ptr(out, np.float64, dev), int(dev))
        self._check(self._device_call(call, w, y, out) if dev else call())
        return out

    def gn_hessvec(self, w, p):
        """Gauss-Newton product (I + G^T G) p of every local problem at w
        (packed control layout)."""
        self._fwd_token += 1
        dev = _is_torch_cuda(w)
        if dev:
            import torch
            out = torch.empty(self.ctrl_total, dtype=torch.float64, device=w.device)
        else:
            w = np.ascontiguousarray(w, dtype=np.float64)
            p = np.ascontiguousarray(p, dtype=np.float64)
            out = np.zeros(self.ctrl_total)
        call = lambda: lib.dd4dv_gn_hessvec(self._h, _ptr(w, np.float64, dev), _ptr(p, np.float64, dev),
                                            _ptr(out, np.float64, dev), int(dev))
        self._check(self._device_call(call, w, p, out) if dev else call())
        return out

    def trajectories(self, w):
        self._fwd_token += 1
        dev = _is_torch_cuda(w)
        if dev:
            import torch
            out = torch.empty(self.traj_total, dtype=torch.float64, device=w.device)
        else:
            w = np.ascontiguousarray(w, dtype=np.float64)
            out = np.zeros(self.traj_total)
        call = lambda: lib.dd4dv_trajectories(self._h, _ptr(w, np.float64, dev), _ptr(out, np.float64, dev),
                                              int(dev))
        self._check(self._device_call(call, w, out) if dev else call())
        return out

    def exchange(self, w):
        self._fwd_token += 1
        dev = _is_torch_cuda(w)
        if not dev:
            w = np.ascontiguousarray(w, dtype=np.float64)
        call = lambda: lib.dd4dv_exchange(self._h, _ptr(w, np.float64, dev), int(dev))
        self._check(self._device_call(call, w) if dev else call())

    def reset_exchange(self):
        self._check(lib.dd4dv_reset_exchange(self._h))

    def boundary_trajectory(self) -> np.ndarray:
        out = np.zeros((self.nsteps + 1, 3, self.nlat, self.nlon))
        self._check(lib.dd4dv_boundary_trajectory(self._h, C.c_void_p(out.ctypes.data), 0))
        return out

    def analysis(self) -> np.ndarray:
        out = np.zeros((3, self.nlat, self.nlon))
        self._check(lib.dd4dv_analysis(self._h, C.c_void_p(out.ctypes.data), 0))
        return out

    def forward(self, x0):
        """Global model run from x0 [3, nlat, nlon]: trajectory [nsteps+1, 3,
        nlat, nlon].  A CUDA float64 tensor in gives a device tensor out
        (no host copy); a host array gives a numpy array."""
        if _is_torch_cuda(x0):
            import torch
            x0 = x0.contiguous()
            out = torch.empty((self.nsteps + 1, 3, self.nlat, self.nlon), dtype=torch.float64, device=x0.device)
            call = lambda: lib.dd4dv_forward(self._h, _ptr(x0, np.float64, True), _ptr(out, np.float64, True), 1)
            self._check(self._device_call(call, x0, out))
            return out
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        out = np.zeros((self.nsteps + 1, 3, self.nlat, self.nlon))
        self._check(lib.dd4dv_forward(self._h, C.c_void_p(x0.ctypes.data), C.c_void_p(out.ctypes.data), 0))
        return out

    def observe(self, traj, level, var, fi, fj):
        """H applied to a global trajectory at the given sites.  A CUDA tensor
        trajectory is read in place and gives a device tensor out."""
        if _is_torch_cuda(traj):
            import torch
            dev = traj.device
            traj = traj.contiguous()
            lv = torch.as_tensor(np.asarray(level, dtype=np.int32), device=dev)
            vr = torch.as_tensor(np.asarray(var, dtype=np.int32), device=dev)
            fi_d = torch.as_tensor(np.asarray(fi, dtype=np.float64), device=dev)
            fj_d = torch.as_tensor(np.asarray(fj, dtype=np.float64), device=dev)
            out = torch.empty(len(lv), dtype=torch.float64, device=dev)
            if len(lv) == 0:
                return out
            call = lambda: lib.dd4dv_observe(self._h, _ptr(traj, np.float64, True), len(lv),
                                             _ptr(lv, np.int32, True), _ptr(vr, np.int32, True),
                                             _ptr(fi_d, np.float64, True), _ptr(fj_d, np.float64, True),
                                             _ptr(out, np.float64, True), 1)
            self._check(self._device_call(call, traj, lv, vr, fi_d, fj_d, out))
            return out
        traj = np.ascontiguousarray(traj, dtype=np.float64)
        lv = np.ascontiguousarray(level, dtype=np.int32)
        vr = np.ascontiguousarray(var, dtype=np.int32)
        fi = np.ascontiguousarray(fi, dtype=np.float64)
        fj = np.ascontiguousarray(fj, dtype=np.float64)
        out = np.zeros(len(lv))
        self._check(lib.dd4dv_observe(self._h, C.c_void_p(traj.ctypes.data), len(lv),
                                      C.c_void_p(lv.ctypes.data), C.c_void_p(vr.ctypes.data),
                                      C.c_void_p(fi.ctypes.data), C.c_void_p(fj.ctypes.data),
                                      C.c_void_p(out.ctypes.data), 0))
        return out

    # ---- outer loop (Alg. 1) ----
    # ---- Turkel-Zwas scheme, undecomposed problem (host numpy arrays) ----
    def _state(self, x):
        return np.ascontiguousarray(x, dtype=np.float64)

    def tz_forward(self, p, q, alpha, x0):
        out = np.zeros((self.nsteps + 1, 3, self.nlat, self.nlon))
        self._check(lib.dd4dv_tz_forward(self._h, p, q, alpha, _ptr(self._state(x0), np.float64, False),
                                         C.c_void_p(out.ctypes.data), 0))
        return out

    def tz_tlm(self, p, q, alpha, x0, dx0):
        out = np.zeros((self.nsteps + 1, 3, self.nlat, self.nlon))
        self._check(lib.dd4dv_tz_tlm(self._h, p, q, alpha, _ptr(self._state(x0), np.float64, False),
                                     _ptr(self._state(dx0), np.float64, False), C.c_void_p(out.ctypes.data), 0))
        return out

    def tz_adjoint(self, p, q, alpha, x0, ytraj):
        out = np.zeros((3, self.nlat, self.nlon))
        self._check(lib.dd4dv_tz_adjoint(self._h, p, q, alpha, _ptr(self._state(x0), np.float64, False),
                                         _ptr(self._state(ytraj), np.float64, False), C.c_void_p(out.ctypes.data),
                                         0))
        return out

    def tz_eval(self, p, q, alpha, w):
        J = np.zeros(1)
        g = np.zeros(3 * self.nlat * self.nlon)
        self._check(lib.dd4dv_tz_eval(self._h, p, q, alpha, _ptr(self._state(w), np.float64, False),
                                      C.c_void_p(J.ctypes.data), C.c_void_p(g.ctypes.data), 0))
        return float(J[0]), g

    def set_owned(self, owned=None):
        """Subdomains this context evaluates and solves (n_sub flags; None = all)."""
        if owned is None:
            self._check(lib.dd4dv_set_owned(self._h, None))
            return
        m = np.ascontiguousarray(owned, dtype=np.int32)
        if m.shape != (self.n_sub,):
            raise ValueError(f"owned must have {self.n_sub} entries")
        self._check(lib.dd4dv_set_owned(self._h, C.c_void_p(m.ctypes.data)))

    def local_solve(self, solver=None, stats=None):
        """Batched L-BFGS on the owned subdomains (one outer iteration without the Exchange)."""
        self._fwd_token += 1
        solver = solver or solver_defaults()
        stats = stats if stats is not None else _abi.dd4dv_stats()
        self._check(lib.dd4dv_local_solve(self._h, C.byref(solver), C.byref(stats)))
        return stats

    def outer_step(self, solver=None, stats=None):
        self._fwd_token += 1
        solver = solver or solver_defaults()
        stats = stats if stats is not None else _abi.dd4dv_stats()
        self._check(lib.dd4dv_outer_step(self._h, C.byref(solver), C.byref(stats)))
        return stats

    def run(self, solver=None):
        self._fwd_token += 1
        solver = solver or solver_defaults()
        stats = _abi.dd4dv_stats()
        xa = np.zeros((3, self.nlat, self.nlon))
        st = self._check(lib.dd4dv_run(self._h, C.byref(solver), C.c_void_p(xa.ctypes.data), C.byref(stats)),
                         allow_notconv=True)
        return xa, stats, st

    def get_controls(self, out=None):
        dev = out is not None and _is_torch_cuda(out)
        w = out if out is not None else np.zeros(self.ctrl_total)
        call = lambda: lib.dd4dv_get_controls(self._h, _ptr(w, np.float64, dev), int(dev))
        self._check(self._device_call(call, w) if dev else call())
        return w

    def set_controls(self, w):
        dev = _is_torch_cuda(w)
        if not dev:
            w = np.ascontiguousarray(w, dtype=np.float64)
        call = lambda: lib.dd4dv_set_controls(self._h, _ptr(w, np.float64, dev), int(dev))
        self._check(self._device_call(call, w) if dev else call())

    # ---- packed-layout helpers ----
    def split_controls(self, w) -> list:
        return [w[self.offsets[s]:self.offsets[s + 1]] for s in range(self.n_sub)]

    def split_traj(self, x) -> list:
        out = []
        for s in range(self.n_sub):
            i0, nx, j0, ny, a, b = self.boxes[s]
            out.append(x[self.traj_offsets[s]:self.traj_offsets[s + 1]].reshape(b - a + 1, 3, ny, nx))
        return out
