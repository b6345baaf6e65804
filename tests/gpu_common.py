"""Shared helpers of the GPU parity tests: move oracle states into the CUDA
library through the C-ABI and compare what comes back.  Pure marshalling: no
arithmetic of the method lives here."""
from __future__ import annotations

import numpy as np

W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
W7 = np.array([0.25] + [0.125] * 6)


def require_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test run without a CUDA device")
    return torch


def make_pair(orc, cfg, Fext=None, storage="f32", **gpu_kw):
    """Oracle solver and CUDA solver with the same parameters.  Fext is
    [3, nz, ny, nx] (float64) or None."""
    from paper_0809_4730_gb300.glbe import Solver
    torch = require_cuda()
    S = orc.Solver(cfg, Fext=None if Fext is None else Fext.reshape(3, -1).T.copy())
    kw = dict(wall_lo=cfg.wall_lo, wall_hi=cfg.wall_hi, rho0=cfg.rho0, gamma=cfg.gamma, nu=cfg.nu, s=cfg.s,
              F=cfg.F, induction=int(cfg.induction), storage=storage)
    if cfg.induction:
        kw.update(gamma_m=cfg.gamma_m, eta=cfg.eta, chi=cfg.chi, mu=cfg.mu, B0=cfg.B0)
    if Fext is not None:
        kw["force_field"] = 3
    kw.update(gpu_kw)
    G = Solver(cfg.nx, cfg.ny, cfg.nz, **kw)
    if Fext is not None:
        G.set_force(torch.tensor(Fext.reshape(3, -1), dtype=torch.float32, device="cuda"))
    return S, G


def push_oracle_state(S, G, t=0):
    """Copies the oracle's (f, g, F_L) into the CUDA context as deviations."""
    torch = require_cuda()
    cfg = S.cfg
    df = (S.f - W19[None, :] * cfg.rho0).T.copy()                  # [19, N]
    dft = torch.tensor(df, dtype=torch.float32, device="cuda")
    dgt = FLt = None
    if cfg.induction:
        B0 = np.asarray(cfg.B0, dtype=float)
        dg = S.g - W7[None, None, :] * B0[None, :, None]              # [N, 3, 7]
        dgt = torch.tensor(dg.reshape(cfg.N, 21).T.copy(), dtype=torch.float32, device="cuda")
        FLt = torch.tensor(S.FL.T.copy(), dtype=torch.float32, device="cuda")
    G.set_state(dft, dgt, FLt, t=t)


def oracle_state_dev(S):
    """Oracle state as deviations in the C-ABI layout (float64)."""
    cfg = S.cfg
    df = (S.f - W19[None, :] * cfg.rho0).T
    dg = FL = None
    if cfg.induction:
        B0 = np.asarray(cfg.B0, dtype=float)
        dg = (S.g - W7[None, None, :] * B0[None, :, None]).reshape(cfg.N, 21).T
        FL = S.FL.T
    return df, dg, FL


def gpu_state(G):
    df, dg, FL = G.get_state()
    G.sync()
    return (df.cpu().double().numpy(), None if dg is None else dg.cpu().double().numpy(),
            None if FL is None else FL.cpu().double().numpy())


def gpu_fields(G):
    rho, u, B = G.fields()
    G.sync()
    return rho.cpu().double().numpy(), u.cpu().double().numpy(), None if B is None else B.cpu().double().numpy()


def rel_linf(a, b, mask=None):
    """max |a - b| / max |b| over the masked entries (columns = nodes)."""
    if mask is not None:
        a = a[..., mask]
        b = b[..., mask]
    scale = np.abs(b).max()
    return np.abs(a - b).max() / (scale if scale > 0 else 1.0)
