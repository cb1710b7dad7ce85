"""Python binding of libosb (ctypes).  Argument marshalling only: every step of
the time step runs in the library's CUDA kernels.  PyTorch supplies the device
buffers and the stream.

The library must be built (``python -m paper_1609_01277_gb300.build`` or
``__graft_entry__.build()``); importing this module on a machine without it
raises, and nothing here falls back to a CPU path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

OSB_FP64, OSB_FP32, OSB_DF64 = 0, 1, 2
OSB_VISC_A, OSB_VISC_B = 0, 1
OSB_BC_PERIODIC, OSB_BC_SYMMETRIC = 0, 1
STATUS = {0: "OSB_OK", 1: "OSB_ERR_INVALID_ARG", 2: "OSB_ERR_UNSUPPORTED", 3: "OSB_ERR_CUDA",
          4: "OSB_ERR_NONFINITE", 5: "OSB_ERR_TIMEOUT", 6: "OSB_ERR_BUFFER", 7: "OSB_ERR_BOUNDS"}

# every entry point declared in include/osb.h
EXPORTS = ("osb_state_bytes", "osb_workspace_bytes", "osb_grid_create", "osb_grid_destroy",
           "osb_init_taylor_green", "osb_set_state", "osb_get_state", "osb_set_state_device",
           "osb_euler_step",
           "osb_get_state_device", "osb_residual", "osb_rk3_step", "osb_diagnostics",
           "osb_batch_step", "osb_batch_configure", "osb_autotune", "osb_autotune_batch", "osb_tile_depth",
           "osb_diagnostics_noalloc",
           "osb_closure_param_count", "osb_closure_workspace_bytes", "osb_closure_create", "osb_closure_destroy",
           "osb_closure_set_normalization", "osb_closure_set_channels", "osb_closure_set_dissipative", "osb_closure_set_loss_weight", "osb_closure_status", "osb_closure_sync_weights",
           "osb_closure_forward", "osb_closure_loss_grad", "osb_closure_adam_step", "osb_grid_set_closure",
           "osb_box_filter", "osb_scalar_rk3", "osb_set_boundaries", "osb_set_diag_series",
           "osb_diag_series_count", "osb_profile_start", "osb_profile_stop", "osb_fp64_rate_probe",
           "osb_set_z_slab", "osb_halo_bytes", "osb_halo_pack", "osb_halo_unpack", "osb_rk3_stage",
           "osb_status_string", "osb_last_error")
KERNEL_KINDS = ("prim", "grad", "resid")


class OsbError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("order", ctypes.c_int), ("precision", ctypes.c_int), ("visc_form", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("Re", ctypes.c_double), ("Mach", ctypes.c_double), ("gamma", ctypes.c_double),
                ("Pr", ctypes.c_double), ("dt", ctypes.c_double)]


class Diag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("step", ctypes.c_longlong), ("ke", ctypes.c_double),
                ("enstrophy", ctypes.c_double), ("total", ctypes.c_double * 5),
                ("nonfinite", ctypes.c_longlong), ("max_cfl", ctypes.c_double)]


_lib = None


def load(path: str | None = None):
    """Load libosb and declare the signatures.  Raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libosb is not built ({path}); run paper_1609_01277_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, sz, dp = ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)
    D, P = ctypes.POINTER(GridDesc), ctypes.POINTER(Params)
    L.osb_state_bytes.argtypes = [D]
    L.osb_state_bytes.restype = sz
    L.osb_workspace_bytes.argtypes = [D]
    L.osb_workspace_bytes.restype = sz
    L.osb_grid_create.argtypes = [D, P, vp, sz, vp, sz, vp, ctypes.POINTER(vp)]
    L.osb_grid_destroy.argtypes = [vp]
    L.osb_init_taylor_green.argtypes = [vp, vp, ctypes.c_double]
    L.osb_set_state.argtypes = [vp, vp]
    L.osb_get_state.argtypes = [vp, vp]
    L.osb_set_state_device.argtypes = [vp, vp]
    L.osb_get_state_device.argtypes = [vp, vp]
    L.osb_residual.argtypes = [vp, vp]
    L.osb_rk3_step.argtypes = [vp, ctypes.c_int]
    L.osb_euler_step.argtypes = [vp, ctypes.c_int]
    L.osb_diagnostics.argtypes = [vp, ctypes.POINTER(Diag)]
    L.osb_batch_step.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int]
    L.osb_batch_configure.argtypes = [ctypes.c_double, ctypes.c_int]
    L.osb_autotune.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.osb_autotune_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int]
    L.osb_tile_depth.argtypes = [ctypes.c_void_p]
    L.osb_tile_depth.restype = ctypes.c_int
    L.osb_diagnostics_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, vp, vp]
    L.osb_scalar_rk3.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int, vp]
    L.osb_set_boundaries.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.osb_set_diag_series.argtypes = [vp, vp, ctypes.c_int]
    L.osb_diag_series_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.osb_profile_start.argtypes = [vp, ctypes.c_int]
    L.osb_profile_stop.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_longlong)]
    L.osb_fp64_rate_probe.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
    L.osb_set_z_slab.argtypes = [vp, ctypes.c_int]
    L.osb_halo_bytes.argtypes = [vp]
    L.osb_halo_bytes.restype = sz
    L.osb_halo_pack.argtypes = [vp, ctypes.c_int, vp, vp]
    L.osb_halo_unpack.argtypes = [vp, ctypes.c_int, vp, vp]
    L.osb_rk3_stage.argtypes = [vp, ctypes.c_int]
    L.osb_status_string.argtypes = [ctypes.c_int]
    L.osb_status_string.restype = ctypes.c_char_p
    L.osb_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("osb_state_bytes", "osb_workspace_bytes", "osb_status_string", "osb_last_error",
                        "osb_closure_param_count", "osb_closure_workspace_bytes", "osb_halo_bytes"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(status: int, where: str) -> None:
    if status != 0:
        raise OsbError(status, where, load().osb_last_error().decode())


@dataclass
class Config:
    nx: int
    ny: int
    nz: int
    order: int = 4
    precision: int = OSB_FP64
    visc_form: int = OSB_VISC_A
    Re: float = 1600.0
    Mach: float = 0.1
    gamma: float = 1.4
    Pr: float = 0.71
    dt: float = 3.385e-3
    # boundary kind per axis (x, y, z): OSB_BC_PERIODIC, or OSB_BC_SYMMETRIC
    # (symmetry planes at 0 and pi, points at (i + 1/2) pi / n)
    bc: tuple = (OSB_BC_PERIODIC, OSB_BC_PERIODIC, OSB_BC_PERIODIC)

    def desc(self) -> GridDesc:
        return GridDesc(self.nx, self.ny, self.nz, self.order, self.precision, self.visc_form)

    def params(self) -> Params:
        return Params(self.Re, self.Mach, self.gamma, self.Pr, self.dt)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (5, self.nz, self.ny, self.nx)


class Grid:
    """One grid on the current CUDA device, advanced on one stream; periodic,
    or with symmetry planes on the axes that ``cfg.bc`` marks."""

    def __init__(self, cfg: Config, stream=None, device=None):
        import torch
        L = load()
        self.cfg = cfg
        self._torch = torch
        device = torch.device(device or "cuda")
        d = cfg.desc()
        sb = L.osb_state_bytes(ctypes.byref(d))
        wb = L.osb_workspace_bytes(ctypes.byref(d))
        if sb == 0 or wb == 0:
            raise OsbError(1, "osb_*_bytes", "invalid grid descriptor")
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.state = torch.empty(sb, dtype=torch.uint8, device=device)
        self.workspace = torch.empty(wb, dtype=torch.uint8, device=device)
        h = ctypes.c_void_p()
        p = cfg.params()
        check(L.osb_grid_create(ctypes.byref(d), ctypes.byref(p), self.state.data_ptr(), sb,
                                self.workspace.data_ptr(), wb, self.stream.cuda_stream, ctypes.byref(h)),
              "osb_grid_create")
        self.handle = h
        if any(b != OSB_BC_PERIODIC for b in cfg.bc):
            check(L.osb_set_boundaries(h, *[int(b) for b in cfg.bc]), "osb_set_boundaries")

    def close(self):
        if getattr(self, "handle", None):
            load().osb_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state ----------------------------------------------------------------
    def init_taylor_green(self, noise=None, amp: float = 0.0) -> None:
        """noise: None, or a (3, nz, ny, nx) float64 array (numpy or CUDA tensor)."""
        torch = self._torch
        ptr = None
        if noise is not None:
            t = torch.as_tensor(noise, dtype=torch.float64)
            t = t.to(self.state.device).contiguous()
            if t.numel() != 3 * self.cfg.n:
                raise ValueError("noise must hold 3*N values")
            self._noise = t  # keep alive until the kernel has run
            ptr = t.data_ptr()
        check(load().osb_init_taylor_green(self.handle, ptr, float(amp)), "osb_init_taylor_green")

    def set_state(self, Q: np.ndarray) -> None:
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        if Q.size != 5 * self.cfg.n:
            raise ValueError("state must hold 5*N values")
        check(load().osb_set_state(self.handle, Q.ctypes.data), "osb_set_state")

    def get_state(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.cfg.shape, dtype=np.float64)
        check(load().osb_get_state(self.handle, out.ctypes.data), "osb_get_state")
        return out

    def set_state_device(self, Q) -> None:
        self._src = Q.contiguous()
        check(load().osb_set_state_device(self.handle, self._src.data_ptr()), "osb_set_state_device")

    def get_state_device(self, out=None):
        torch = self._torch
        if out is None:
            out = torch.empty(self.cfg.shape, dtype=torch.float64, device=self.state.device)
        check(load().osb_get_state_device(self.handle, out.data_ptr()), "osb_get_state_device")
        return out

    # -- compute --------------------------------------------------------------
    def residual(self, out=None):
        torch = self._torch
        if out is None:
            out = torch.empty(self.cfg.shape, dtype=torch.float64, device=self.state.device)
        check(load().osb_residual(self.handle, out.data_ptr()), "osb_residual")
        return out

    def step(self, nsteps: int = 1) -> None:
        check(load().osb_rk3_step(self.handle, int(nsteps)), "osb_rk3_step")

    def stage(self, k: int) -> None:
        """RK stage k (0, 1, 2 in order) of the step in progress."""
        check(load().osb_rk3_stage(self.handle, int(k)), "osb_rk3_stage")

    def set_z_slab(self, nz_domain: int) -> None:
        """Make this grid a z-slab (ghost planes included in nz) of a periodic
        box of nz_domain planes."""
        check(load().osb_set_z_slab(self.handle, int(nz_domain)), "osb_set_z_slab")

    def halo_bytes(self) -> int:
        return int(load().osb_halo_bytes(self.handle))

    def halo_pack(self, source: int, send_lo, send_hi) -> None:
        """Pack the planes next to the slab faces of a source (0..2: stage
        source, 3: accumulator) into two device buffers (torch tensors)."""
        check(load().osb_halo_pack(self.handle, int(source), send_lo.data_ptr(), send_hi.data_ptr()),
              "osb_halo_pack")

    def halo_unpack(self, source: int, recv_lo, recv_hi) -> None:
        check(load().osb_halo_unpack(self.handle, int(source), recv_lo.data_ptr(), recv_hi.data_ptr()),
              "osb_halo_unpack")

    def euler_step(self, nsteps: int = 1) -> None:
        """Forward Euler steps (Section 2.4), mixable with step()."""
        check(load().osb_euler_step(self.handle, int(nsteps)), "osb_euler_step")

    def set_diag_series(self, capacity: int | None) -> None:
        """Record the kinetic energy and enstrophy of the state at the start of
        every step (fused into the first stage) into a device ring of
        ``capacity`` entries; None stops recording."""
        torch = self._torch
        if capacity is None:
            check(load().osb_set_diag_series(self.handle, None, 0), "osb_set_diag_series")
            self._series = None
            return
        self._series = torch.zeros(2 * int(capacity), dtype=torch.float64, device=self.state.device)
        check(load().osb_set_diag_series(self.handle, self._series.data_ptr(), int(capacity)), "osb_set_diag_series")

    def diag_series(self) -> np.ndarray:
        """(steps, 2) array of (ke, enstrophy), oldest first (the last
        ``capacity`` steps once the ring has wrapped)."""
        n = ctypes.c_longlong()
        check(load().osb_diag_series_count(self.handle, ctypes.byref(n)), "osb_diag_series_count")
        buf = self._series.cpu().numpy().reshape(-1, 2)
        cap = buf.shape[0]
        k = int(n.value)
        if k <= cap:
            return buf[:k].copy()
        start = k % cap
        return np.concatenate([buf[start:], buf[:start]])

    def profile_start(self, max_stages: int) -> None:
        check(load().osb_profile_start(self.handle, int(max_stages)), "osb_profile_start")

    def profile_stop(self) -> dict:
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_longlong * 3)()
        check(load().osb_profile_stop(self.handle, ms, n), "osb_profile_stop")
        return {k: dict(total_ms=ms[i], launches=n[i]) for i, k in enumerate(KERNEL_KINDS)}

    def diagnostics(self, raise_nonfinite: bool = True) -> dict:
        d = Diag()
        st = load().osb_diagnostics(self.handle, ctypes.byref(d))
        if st != 0 and (raise_nonfinite or st != 4):
            check(st, "osb_diagnostics")
        return dict(t=d.t, step=d.step, ke=d.ke, enstrophy=d.enstrophy, total=list(d.total),
                    nonfinite=d.nonfinite, max_cfl=d.max_cfl, status=st)


def diagnostics_noalloc(Q_dev, cfg: Config, out_dev, stream=None) -> None:
    """Diagnostics of a caller-owned device state (5*N FP64, no padding) into a
    caller-owned device array of 9 FP64 values, with no device allocation
    (for callers that cannot allocate at that point, e.g. during a global-mode
    stream capture).  Stream-ordered; the caller synchronises."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    p = cfg.params()
    check(load().osb_diagnostics_noalloc(Q_dev.data_ptr(), cfg.nx, cfg.ny, cfg.nz, cfg.order, ctypes.byref(p),
                                         out_dev.data_ptr(), st.cuda_stream), "osb_diagnostics_noalloc")


def scalar_rk3(phi, work, order: int, adv=(0.0, 0.0, 0.0), diff: float = 0.0, dt: float = 1e-3,
               nsteps: int = 1, src=None, stream=None) -> None:
    """Advance the scalar field phi (a (nz, ny, nx) float64 CUDA tensor, in place)
    by nsteps RK3 steps of d phi/dt = -a_j D_j phi + k L_j phi - S on the
    periodic box [0, 2 pi)^3 (paper Sections 3.1-3.2).  work: a CUDA float64
    tensor of at least 2 * phi.numel() values; src: None or a tensor like phi."""
    import torch
    if phi.dtype != torch.float64 or not phi.is_cuda or not phi.is_contiguous() or phi.dim() != 3:
        raise ValueError("phi must be a contiguous (nz, ny, nx) float64 CUDA tensor")
    if work.dtype != torch.float64 or not work.is_cuda or work.numel() < 2 * phi.numel():
        raise ValueError("work must be a float64 CUDA tensor of 2 * phi.numel() values")
    if src is not None and (src.dtype != torch.float64 or not src.is_cuda or src.shape != phi.shape
                            or not src.is_contiguous()):
        raise ValueError("src must be a contiguous float64 CUDA tensor shaped like phi")
    st = stream if stream is not None else torch.cuda.current_stream()
    nz, ny, nx = phi.shape
    a = (ctypes.c_double * 3)(*[float(v) for v in adv])
    check(load().osb_scalar_rk3(phi.data_ptr(), work.data_ptr(), None if src is None else src.data_ptr(),
                                nx, ny, nz, int(order), a, float(diff), float(dt), int(nsteps), st.cuda_stream),
          "osb_scalar_rk3")


def batch_step(grids, nsteps: int) -> None:
    """Advances every grid nsteps steps: FP64 and FP32 in one persistent,
    graph-captured launch; double-float as each grid's step graph on
    concurrent library streams (OSB_BATCH_MODE overrides)."""
    arr = (ctypes.c_void_p * len(grids))(*[g.handle for g in grids])
    check(load().osb_batch_step(arr, len(grids), int(nsteps)), "osb_batch_step")


def batch_configure(wait_limit_seconds: float = 2.0, test_stall: bool = False) -> None:
    check(load().osb_batch_configure(float(wait_limit_seconds), int(bool(test_stall))), "osb_batch_configure")


def autotune(grid: "Grid", trial_steps: int = 3) -> int:
    """Pick the ensemble tile depth for this grid's shape (state is restored)."""
    tz = ctypes.c_int(0)
    check(load().osb_autotune(grid.handle, int(trial_steps), ctypes.byref(tz)), "osb_autotune")
    return tz.value


def autotune_batch(grids, trial_steps: int = 2) -> dict:
    """Tune the persistent kernel's tile depth of every grid shape in the
    ensemble, timed on the whole ensemble (states restored); returns
    {shape: depth}."""
    arr = (ctypes.c_void_p * len(grids))(*[g.handle for g in grids])
    check(load().osb_autotune_batch(arr, len(grids), int(trial_steps)), "osb_autotune_batch")
    out = {}
    for g in grids:
        out[(g.cfg.nx, g.cfg.ny, g.cfg.nz)] = tile_depth(g.cfg)
    return out


def tile_depth(cfg: "Config") -> int:
    """Tile depth (z planes per work item) the ensemble kernel uses for this shape."""
    d = cfg.desc() if hasattr(cfg, "desc") else cfg
    return int(load().osb_tile_depth(ctypes.byref(d)))


def fp64_rate(blocks: int = 152 * 8, iters: int = 2000, repeats: int = 5) -> dict:
    """Measured FP64 fused multiply-add rate (TFLOP/s): the library's probe
    kernel timed with CUDA events on the stream it runs on, after a warm-up
    launch; the best of `repeats` launches."""
    import torch
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    L = load()
    check(L.osb_fp64_rate_probe(out.data_ptr(), blocks, iters, st.cuda_stream), "osb_fp64_rate_probe")
    best = None
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        check(L.osb_fp64_rate_probe(out.data_ptr(), blocks, iters, st.cuda_stream), "osb_fp64_rate_probe")
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    flops = blocks * 256 * 8 * 16 * iters * 2
    return {"tflops": flops / (best * 1e-3) / 1e12, "ms": best, "blocks": blocks, "iters": iters,
            "flops": flops}
