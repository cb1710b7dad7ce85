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
    L.osb_closure_set_channels.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.osb_closure_set_dissipative.argtypes = [vp, ctypes.c_int]
    L.osb_closure_set_loss_weight.argtypes = [vp, ctypes.c_float]
    L.osb_closure_status.argtypes = [vp]
    L.osb_closure_forward.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.osb_closure_loss_grad.argtypes = [vp, vp, ctypes.c_size_t, vp, ctypes.c_size_t, vp, vp]
    L.osb_closure_adam_step.argtypes = [vp, vp, ctypes.c_float, ctypes.c_int]
    L.osb_grid_set_closure.argtypes = [vp, vp]
    L.osb_box_filter.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    for name in ("osb_closure_create", "osb_closure_destroy", "osb_closure_set_normalization",
                 "osb_closure_sync_weights", "osb_closure_set_channels", "osb_closure_set_dissipative",
                 "osb_closure_set_loss_weight",
                 "osb_closure_status", "osb_closure_forward", "osb_closure_loss_grad",
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

    def status(self) -> None:
        check(_declare().osb_closure_status(self.handle), "osb_closure_status")

    def set_channels(self, apply) -> None:
        arr = (ctypes.c_int * 5)(*[int(bool(v)) for v in apply])
        check(_declare().osb_closure_set_channels(self.handle, arr), "osb_closure_set_channels")

    def set_loss_weight(self, w: float) -> None:
        check(_declare().osb_closure_set_loss_weight(self.handle, float(w)), "osb_closure_set_loss_weight")

    def set_dissipative(self, on: bool) -> None:
        """Clip the momentum correction's local kinetic-energy injection."""
        check(_declare().osb_closure_set_dissipative(self.handle, int(bool(on))), "osb_closure_set_dissipative")

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


def train(closure: Closure, data, epochs: int, lr: float = 1e-3, train_idx=None, seed: int = 0,
          relative: bool = False):
    """Adam over the snapshots in random order.  relative: weight each
    snapshot's loss by the inverse mean square of its normalised target (mean
    weight 1), so snapshots with a small commutation residual -- the smooth
    early flow -- are fitted in relative terms too."""
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = list(range(len(data["X"]))) if train_idx is None else list(train_idx)
    weights = {i: 1.0 for i in idx}
    if relative:
        import torch
        out_std = torch.tensor(np.asarray(closure.norm[2], dtype=np.float64), device=data["Y"][0].device).view(5, 1, 1, 1)
        ms = {i: float(((data["Y"][i] / out_std) ** 2).mean()) for i in idx}
        inv = {i: 1.0 / max(ms[i], 1e-30) for i in idx}
        mean_inv = float(np.mean(list(inv.values())))
        weights = {i: inv[i] / mean_inv for i in idx}
    hist = []
    for _ in range(epochs):
        order = rng.permutation(idx)
        tot = 0.0
        for i in order:
            closure.set_loss_weight(weights[int(i)])
            tot += float(closure.train_step(data["X"][i], data["Y"][i], lr).item())
        hist.append(tot / len(order))
    closure.set_loss_weight(1.0)
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


def _ke_run(grid, X0, steps_per_sample, samples, closure=None, history=4):
    """KE of a coarse run every steps_per_sample steps (from state X0).

    With a closure attached, the plain solver is the fallback: when a sample
    shows the signs that precede a blow-up -- a non-finite state, kinetic energy
    above 1.01 E_k(0) (the decaying Taylor-Green flow never gains energy), or a
    Courant number above twice its initial value -- the run returns to the
    oldest of the last `history` good samples, detaches the closure and
    continues from there with the plain solver.
    Returns (ke, seconds, fallback_time or None)."""
    import time

    import torch
    grid.set_state_device(X0)
    if closure is not None:
        closure.attach(grid)
    d0 = grid.diagnostics()
    ke = [d0["ke"]]
    hist = [(0, grid.get_state_device().clone())] if closure is not None else []
    fallback_t = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = 0
    while s < samples - 1:
        grid.step(steps_per_sample)
        s += 1
        d = grid.diagnostics(raise_nonfinite=False)
        if closure is not None and fallback_t is None:
            if (d["status"] != 0 or not np.isfinite(d["ke"]) or d["ke"] > 1.01 * d0["ke"]
                    or not d["max_cfl"] < 2.0 * d0["max_cfl"]):
                s0, good = hist[0]
                fallback_t = s0 * steps_per_sample * grid.cfg.dt
                Closure.detach(grid)
                grid.set_state_device(good)
                del ke[s0 + 1:]
                s = s0
                continue
            hist.append((s, grid.get_state_device().clone()))
            if len(hist) > history:
                hist.pop(0)
        ke.append(d["ke"])
    el = time.perf_counter() - t0
    if closure is not None and fallback_t is None:
        Closure.detach(grid)
    return np.array(ke), el, fallback_t


def run_experiment(n_fine=256, factor=4, t_end=10.0, snap_every=48, epochs=20, lr=1e-3, Re=1600.0, order=4,
                   seed=0, relative=False):
    """Fine run -> filtered training data -> training -> a-posteriori KE-decay
    comparison of the coarse grid with and without the closure (and the plain
    solver at twice the coarse resolution), against the filtered fine run."""
    import time

    import torch
    n_c = n_fine // factor
    dt_f = 3.385e-3 * 64.0 / n_fine
    samples = int(round(t_end / (snap_every * dt_f))) + 1
    t0 = time.perf_counter()
    data = make_training_data(n_fine, factor, samples, snap_every, order=order, Re=Re, dt_fine=dt_f)
    t_data = time.perf_counter() - t0
    times = np.array(data["t"])
    # reference: KE of the filtered fine state (coarse-grid diagnostics)
    ref_grid = osb.Grid(osb.Config(n_c, n_c, n_c, order=order, Re=Re, dt=dt_f * factor))
    ke_ref = []
    for X in data["X"]:
        ref_grid.set_state_device(X)
        ke_ref.append(ref_grid.diagnostics()["ke"])
    ke_ref = np.array(ke_ref)
    ke_fine = np.array(data["ke_fine"])
    # training on 3 of every 4 snapshots
    train_idx = [i for i in range(samples) if i % 4 != 3]
    test_idx = [i for i in range(samples) if i % 4 == 3]
    c = Closure(n_c, n_c, n_c, seed=seed)
    c.set_normalization(*normalisation(data))
    t0 = time.perf_counter()
    hist = train(c, data, epochs, lr=lr, train_idx=train_idx, seed=seed, relative=relative)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    apriori = dict(plain=a_priori_error(None, data, test_idx), closure=a_priori_error(c, data, test_idx))
    # a posteriori: coarse runs from the filtered initial state
    cstep = snap_every // factor
    g = osb.Grid(osb.Config(n_c, n_c, n_c, order=order, Re=Re, dt=dt_f * factor))
    ke_plain, t_plain, _ = _ke_run(g, data["X"][0], cstep, samples)
    gains = {}
    in_mean, in_std, out_std = c.norm
    for label, apply, gain, diss in (("momentum", (0, 1, 1, 1, 0), 1.0, False),
                                     ("momentum_half", (0, 1, 1, 1, 0), 0.5, False),
                                     ("momentum_dissipative", (0, 1, 1, 1, 0), 1.0, True),
                                     ("momentum_half_dissipative", (0, 1, 1, 1, 0), 0.5, True),
                                     ("all", (1, 1, 1, 1, 1), 1.0, False)):
        c.set_channels(apply)
        c.set_normalization(in_mean, in_std, out_std * gain)
        c.set_dissipative(diss)
        gains[label] = _ke_run(g, data["X"][0], cstep, samples, closure=c)
    c.set_dissipative(False)
    # default for later use: momentum equations only, half gain
    c.set_normalization(in_mean, in_std, out_std * 0.5)
    c.set_channels((0, 1, 1, 1, 0))
    # plain solver at twice the coarse resolution, started from the factor/2 filtered fine state
    n2 = 2 * n_c
    g2 = osb.Grid(osb.Config(n2, n2, n2, order=order, Re=Re, dt=dt_f * factor / 2))
    fine0 = osb.Grid(osb.Config(n_fine, n_fine, n_fine, order=order, Re=Re, dt=dt_f))
    from . import inputs
    fine0.init_taylor_green(torch.from_numpy(inputs.gaussian_noise(n_fine, n_fine, n_fine, 1234)).cuda(), 1e-4)
    X2 = box_filter(fine0.get_state_device(), (n_fine,) * 3, factor // 2)
    del fine0
    ke_2x, t_2x, _ = _ke_run(g2, X2, 2 * cstep, samples)

    def err(ke, ref):
        return float(np.max(np.abs(ke - ref)) / ref[0])

    def eps(ke):
        return -np.gradient(ke, times)

    def eps_err(ke, ref):
        e, r = eps(ke), eps(ref)
        return float(np.max(np.abs(e - r)) / np.max(np.abs(r)))

    res = dict(n_fine=n_fine, factor=factor, n_coarse=n_c, t_end=float(times[-1]), samples=samples,
               snap_every_fine_steps=snap_every, epochs=epochs, train_snapshots=len(train_idx),
               loss_first=hist[0], loss_last=hist[-1], a_priori_rel_err=apriori,
               plain=dict(ke_err_vs_filtered_fine=err(ke_plain, ke_ref), ke_err_vs_fine=err(ke_plain, ke_fine),
                          dissipation_err=eps_err(ke_plain, ke_ref), seconds=t_plain),
               plain_2x=dict(ke_err_vs_filtered_fine=err(ke_2x, ke_ref), ke_err_vs_fine=err(ke_2x, ke_fine),
                             dissipation_err=eps_err(ke_2x, ke_ref), seconds=t_2x),
               closure={label: dict(ke_err_vs_filtered_fine=err(v[0], ke_ref), ke_err_vs_fine=err(v[0], ke_fine),
                                        dissipation_err=eps_err(v[0], ke_ref), seconds=v[1], fallback_t=v[2])
                        for label, v in gains.items()},
               seconds=dict(fine_data=t_data, train=t_train),
               curves=dict(t=times.tolist(), ke_filtered_fine=ke_ref.tolist(), ke_fine=ke_fine.tolist(),
                           ke_plain=ke_plain.tolist(), ke_plain_2x=ke_2x.tolist(),
                           **{f"ke_closure_{label}": v[0].tolist() for label, v in gains.items()}))
    return res


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="learned-closure experiment on the Taylor-Green vortex")
    ap.add_argument("--fine", type=int, default=256)
    ap.add_argument("--factor", type=int, default=4)
    ap.add_argument("--t-end", type=float, default=10.0)
    ap.add_argument("--snap-every", type=int, default=48)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=None)
    ap.add_argument("--relative", action="store_true", help="weight each snapshot by its inverse mean-square target")
    a = ap.parse_args()
    from . import build
    build.build()
    osb.load()
    r = run_experiment(a.fine, a.factor, a.t_end, a.snap_every, a.epochs, a.lr, relative=a.relative)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f)
    print(json.dumps({k: v for k, v in r.items() if k != "curves"}))
