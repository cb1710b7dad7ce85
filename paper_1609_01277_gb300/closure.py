"""Learned residual correction ("closure") for coarse grids: binding and the
training / evaluation driver.  Every arithmetic step (box filter, residuals,
network forward and backward, Adam) runs in libosb's CUDA kernels; this module
allocates device memory through PyTorch and sequences the calls.

Training data are made by the solver itself: a fine run is box-filtered onto
the coarse grid, and the target is the commutation residual
    C* = F(R_fine(Q_f)) - R_coarse(F(Q_f)),
the part of the filtered fine dynamics the coarse discretisation misses.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import osb
from .osb import check, load

NPARAM = 36357


def _declare():
    L = load()
    if getattr(L, "_closure_declared", False):
        return L
    vp, dp, fp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
    L.osb_closure_param_count.restype = ctypes.c_size_t
    L.osb_closure_workspace_bytes.argtypes = [ctypes.c_int] * 3
    L.osb_closure_workspace_bytes.restype = ctypes.c_size_t
    L.osb_closure_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, ctypes.c_size_t, vp,
                                     ctypes.POINTER(vp)]
    L.osb_closure_destroy.argtypes = [vp]
    L.osb_closure_set_normalization.argtypes = [vp, fp, fp, fp]
    L.osb_closure_sync_weights.argtypes = [vp]
    L.osb_closure_forward.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.osb_closure_loss_grad.argtypes = [vp, vp, ctypes.c_size_t, vp, ctypes.c_size_t, vp, vp]
    L.osb_closure_adam_step.argtypes = [vp, vp, ctypes.c_float, ctypes.c_int]
    L.osb_grid_set_closure.argtypes = [vp, vp]
    L.osb_box_filter.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    for name in ("osb_closure_create", "osb_closure_destroy", "osb_closure_set_normalization",
                 "osb_closure_sync_weights", "osb_closure_forward", "osb_closure_loss_grad",
                 "osb_closure_adam_step", "osb_grid_set_closure", "osb_box_filter"):
        getattr(L, name).restype = ctypes.c_int
    L._closure_declared = True
    return L


def init_params(seed: int = 0, scale_out: float = 0.1) -> np.ndarray:
    """He-normal weights (seeded), zero biases; the output layer scaled down so
    that an untrained network adds a small correction."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for name, shape in (("W1", (32, 5, 27)), ("b1", (32,)), ("W2", (32, 32, 27)), ("b2", (32,)),
                        ("W3", (5, 32, 27)), ("b3", (5,))):
        if name[0] == "W":
            fan_in = shape[1] * 27
            w = rng.standard_normal(shape) * np.sqrt(2.0 / fan_in)
            if name == "W3":
                w *= scale_out
            parts.append(w.ravel())
        else:
            parts.append(np.zeros(shape).ravel())
    return np.concatenate(parts).astype(np.float32)


class Closure:
    def __init__(self, nx, ny, nz, stream=None, params: np.ndarray | None = None, seed: int = 0):
        import torch
        L = _declare()
        assert int(L.osb_closure_param_count()) == NPARAM
        self._torch = torch
        self.shape = (nx, ny, nz)
        self.n = nx * ny * nz
        wb = L.osb_closure_workspace_bytes(nx, ny, nz)
        if wb == 0:
            raise osb.OsbError(2, "osb_closure_workspace_bytes", "sizes must be multiples of (8, 4, 4)")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.params = torch.zeros(3 * NPARAM, dtype=torch.float32, device="cuda")
        self.grad = torch.zeros(NPARAM, dtype=torch.float32, device="cuda")
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.workspace = torch.empty(wb, dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        check(L.osb_closure_create(nx, ny, nz, self.params.data_ptr(), self.workspace.data_ptr(), wb,
                                   self.stream.cuda_stream, ctypes.byref(h)), "osb_closure_create")
        self.handle = h
        self.step_count = 0
        self.set_params(init_params(seed) if params is None else params)

    def close(self):
        if getattr(self, "handle", None):
            _declare().osb_closure_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta: np.ndarray) -> None:
        t = self._torch.as_tensor(np.asarray(theta, np.float32)).cuda()
        self.params[:NPARAM].copy_(t)
        self.params[NPARAM:].zero_()
        self.step_count = 0
        check(_declare().osb_closure_sync_weights(self.handle), "osb_closure_sync_weights")

    def get_params(self) -> np.ndarray:
        return self.params[:NPARAM].cpu().numpy().copy()

    def set_normalization(self, in_mean, in_std, out_std) -> None:
        f = lambda a: (ctypes.c_float * 5)(*[float(v) for v in a])  # noqa: E731
        self.norm = (np.asarray(in_mean, float), np.asarray(in_std, float), np.asarray(out_std, float))
        check(_declare().osb_closure_set_normalization(self.handle, f(in_mean), f(in_std), f(out_std)),
              "osb_closure_set_normalization")

    def forward(self, Q_dev):
        """Correction C (5, nz, ny, nx) FP32 for a device FP64 state (5, nz, ny, nx)."""
        torch = self._torch
        nx, ny, nz = self.shape
        C = torch.empty((5, nz, ny, nx), dtype=torch.float32, device="cuda")
        Q = Q_dev.contiguous()
        check(_declare().osb_closure_forward(self.handle, Q.data_ptr(), self.n, C.data_ptr()), "osb_closure_forward")
        return C

    def loss_grad(self, X_dev, Cstar_dev):
        X, Cs = X_dev.contiguous(), Cstar_dev.contiguous()
        check(_declare().osb_closure_loss_grad(self.handle, X.data_ptr(), self.n, Cs.data_ptr(), self.n,
                                               self.grad.data_ptr(), self.loss.data_ptr()), "osb_closure_loss_grad")
        return self.loss, self.grad

    def train_step(self, X_dev, Cstar_dev, lr: float):
        loss, grad = self.loss_grad(X_dev, Cstar_dev)
        self.step_count += 1
        check(_declare().osb_closure_adam_step(self.handle, grad.data_ptr(), float(lr), self.step_count),
              "osb_closure_adam_step")
        return loss

    def attach(self, grid) -> None:
        check(_declare().osb_grid_set_closure(grid.handle, self.handle), "osb_grid_set_closure")
        self._attached = grid

    @staticmethod
    def detach(grid) -> None:
        check(_declare().osb_grid_set_closure(grid.handle, None), "osb_grid_set_closure")


def box_filter(fine_dev, fine_shape, factor: int, stream=None):
    """Box filter of a device FP64 state (5, fnz, fny, fnx) onto (5, fnz/f, fny/f, fnx/f)."""
    import torch
    fnx, fny, fnz = fine_shape
    out = torch.empty((5, fnz // factor, fny // factor, fnx // factor), dtype=torch.float64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    src = fine_dev.contiguous()
    check(_declare().osb_box_filter(src.data_ptr(), fnx, fny, fnz, factor, out.data_ptr(), st.cuda_stream),
          "osb_box_filter")
    return out


# ---------------------------------------------------------------------------
# Data generation, training and evaluation
# ---------------------------------------------------------------------------
def make_training_data(n_fine: int, factor: int, snapshots: int, every: int, order: int = 4, Re: float = 1600.0,
                       Mach: float = 0.1, dt_fine: float | None = None, precision=osb.OSB_FP32, noise_seed: int = 1234):
    """Runs the fine Taylor-Green case, and every `every` steps stores the
    filtered state X = F(Q_f) and the target C* = F(R_f(Q_f)) - R_c(F(Q_f))."""
    import torch
    n_c = n_fine // factor
    dt_f = dt_fine if dt_fine is not None else 3.385e-3 * 64.0 / n_fine
    fine = osb.Grid(osb.Config(n_fine, n_fine, n_fine, order=order, precision=precision, Re=Re, Mach=Mach, dt=dt_f))
    from . import inputs
    fine.init_taylor_green(torch.from_numpy(inputs.gaussian_noise(n_fine, n_fine, n_fine, noise_seed)).cuda(), 1e-4)
    coarse = osb.Grid(osb.Config(n_c, n_c, n_c, order=order, precision=osb.OSB_FP64, Re=Re, Mach=Mach,
                                 dt=dt_f * factor))
    X, Y, T, KE = [], [], [], []
    fine64 = osb.Grid(osb.Config(n_fine, n_fine, n_fine, order=order, precision=osb.OSB_FP64, Re=Re, Mach=Mach,
                                 dt=dt_f))
    for s in range(snapshots):
        if s:
            fine.step(every)
        Qf = fine.get_state_device()
        fine64.set_state_device(Qf)
        Rf = fine64.residual()
        Xc = box_filter(Qf, (n_fine,) * 3, factor)
        Rf_c = box_filter(Rf, (n_fine,) * 3, factor)
        coarse.set_state_device(Xc)
        Rc = coarse.residual()
        X.append(Xc)
        Y.append(Rf_c - Rc)
        T.append(s * every * dt_f)
        KE.append(fine.diagnostics()["ke"])
    torch.cuda.synchronize()
    return dict(X=X, Y=Y, t=T, ke_fine=KE, n_coarse=n_c, dt_coarse=dt_f * factor, order=order, Re=Re, Mach=Mach)


def normalisation(data):
    X = np.stack([x.cpu().numpy() for x in data["X"]])
    Y = np.stack([y.cpu().numpy() for y in data["Y"]])
    in_mean = X.mean(axis=(0, 2, 3, 4))
    in_std = X.std(axis=(0, 2, 3, 4)) + 1e-12
    out_std = Y.std(axis=(0, 2, 3, 4)) + 1e-30
    return in_mean, in_std, out_std


def train(closure: Closure, data, epochs: int, lr: float = 1e-3, train_idx=None, seed: int = 0):
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = list(range(len(data["X"]))) if train_idx is None else list(train_idx)
    hist = []
    for _ in range(epochs):
        order = rng.permutation(idx)
        tot = 0.0
        for i in order:
            tot += float(closure.train_step(data["X"][i], data["Y"][i], lr).item())
        hist.append(tot / len(order))
    return hist


def a_priori_error(closure: Closure | None, data, idx):
    """sum_i ||C*_i - C_i|| / sum_i ||C*_i|| over snapshots idx (C = 0 without a closure)."""
    num = den = 0.0
    for i in idx:
        Y = data["Y"][i]
        C = closure.forward(data["X"][i]).double() if closure is not None else 0.0 * Y
        num += float((Y - C).norm())
        den += float(Y.norm())
    return num / den
