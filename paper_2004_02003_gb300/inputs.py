"""Seeded synthetic inputs: velocity fields on the node grid of a block.

This module generates INPUTS only and holds none of the method's arithmetic
(no interpolation, no integration, no termination). Both the CUDA path and the
oracle receive the same float32 arrays produced here.

The paper's data sets (Cloverleaf3D, Jet, Nyx) are not available; these
fields stand in for them with the shapes of the paper's workloads:

* ``abc_field``: the time-dependent Arnold-Beltrami-Childress flow used in
  the paper's ABC experiment (Sec. 5.2), A = sqrt(3), B = sqrt(2), C = 1,
  with a 0.1*sin(2*pi*t) phase modulation (reading: the modulation shifts the
  argument of every sine and cosine by 0.1*sin(2*pi*t); positions are in
  physical units on [0,1]^3 without a 2*pi rescale).
* ``fourier_field``: divergence-free random Fourier-mode turbulence
  ``u(x, c) = scale * sum_m a_m e_m cos(2 pi k_m . x + phi_m + c delta_m)``,
  |k_m| ~ U[kmin, kmax] with uniform direction, a_m = |k_m|^(-5/6),
  e_m a unit vector perpendicular to k_m (so div u = 0 exactly),
  phi_m ~ U[0, 2 pi), per-cycle phase drift delta_m ~ U[0, drift_max].
  ``scale`` makes max|u| = 1 over a 65^3 lattice of the unit domain at cycle 0.
* ``affine_field`` / ``rotation_field``: closed-form test fields.

Node coordinates are ``origin + i * h`` computed in double from the float32
origin and spacing the library receives.

Evaluation of the Fourier sum uses its separable form: the complex exponential
of 2 pi k.x factors into per-axis terms, so a whole block is two real matrix
products per component instead of a cosine per node and mode.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

ABC_A = float(np.sqrt(3.0))
ABC_B = float(np.sqrt(2.0))
ABC_C = 1.0


def node_coords(n, origin, h):
    """Per-axis node coordinates (float64) of a block with ``n`` cells."""
    o = np.asarray(origin, dtype=np.float32).astype(np.float64)
    hh = np.asarray(h, dtype=np.float32).astype(np.float64)
    return [o[a] + np.arange(int(n[a]) + 1, dtype=np.float64) * hh[a] for a in range(3)]


def _pack(ux, uy, uz):
    return np.ascontiguousarray(np.stack([ux, uy, uz], axis=-1), dtype=np.float32)


def abc_field(n, origin, h, t: float, eps: float = 0.1) -> np.ndarray:
    """ABC flow at time t on the block's nodes; float32 (nz+1, ny+1, nx+1, 3)."""
    x, y, z = node_coords(n, origin, h)
    s = eps * np.sin(2.0 * np.pi * t)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    ux = ABC_A * np.sin(Z + s) + ABC_C * np.cos(Y + s)
    uy = ABC_B * np.sin(X + s) + ABC_A * np.cos(Z + s)
    uz = ABC_C * np.sin(Y + s) + ABC_B * np.cos(X + s)
    return _pack(ux, uy, uz)


def abc_field_torch(n, origin, h, t: float, device, eps: float = 0.1):
    """Same field as :func:`abc_field`, evaluated with torch on ``device`` in
    float64 and rounded to float32."""
    import torch
    x, y, z = (torch.as_tensor(v, dtype=torch.float64, device=device) for v in node_coords(n, origin, h))
    s = eps * np.sin(2.0 * np.pi * t)
    Z, Y, X = torch.meshgrid(z, y, x, indexing="ij")
    ux = ABC_A * torch.sin(Z + s) + ABC_C * torch.cos(Y + s)
    uy = ABC_B * torch.sin(X + s) + ABC_A * torch.cos(Z + s)
    uz = ABC_C * torch.sin(Y + s) + ABC_B * torch.cos(X + s)
    return torch.stack([ux, uy, uz], dim=-1).to(torch.float32).contiguous()


DG_A, DG_EPS, DG_OMEGA = 0.1, 0.25, 2.0 * np.pi / 10.0


def double_gyre_fourier_torch(modes: "FourierModes", n, origin, h, t: float, cycle: int, device,
                              turb: float = 0.1):
    """Double gyre in (x, y) (the Shadden et al. form: stream function
    A sin(pi f(x, t)) sin(pi y), f = a x^2 + b x, a = eps sin(omega t),
    b = 1 - 2 eps sin(omega t), A = 0.1, eps = 0.25, omega = 2 pi / 10, on
    [0, 2] x [0, 1]), constant in z, plus ``turb`` times the Fourier-mode
    turbulence of ``modes`` at ``cycle`` (which supplies the z component).
    Evaluated with torch in float64 on ``device``, rounded to float32."""
    import torch
    x, y, z = (torch.as_tensor(v, dtype=torch.float64, device=device) for v in node_coords(n, origin, h))
    a = DG_EPS * np.sin(DG_OMEGA * t)
    b = 1.0 - 2.0 * DG_EPS * np.sin(DG_OMEGA * t)
    Y, X = torch.meshgrid(y, x, indexing="ij")
    f = a * X * X + b * X
    u = -np.pi * DG_A * torch.sin(np.pi * f) * torch.cos(np.pi * Y)
    v = np.pi * DG_A * torch.cos(np.pi * f) * torch.sin(np.pi * Y) * (2.0 * a * X + b)
    out = turb * fourier_field_torch(modes, n, origin, h, cycle, device).to(torch.float64)
    out[..., 0] += u[None]
    out[..., 1] += v[None]
    return out.to(torch.float32).contiguous()


def uniform_field(n, vel) -> np.ndarray:
    shape = (int(n[2]) + 1, int(n[1]) + 1, int(n[0]) + 1, 3)
    out = np.empty(shape, dtype=np.float32)
    out[...] = np.asarray(vel, dtype=np.float32)
    return out


def affine_field(n, origin, h, A, b) -> np.ndarray:
    """u(x) = A x + b sampled at the nodes (float32)."""
    x, y, z = node_coords(n, origin, h)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    P = np.stack([X, Y, Z], axis=-1)
    U = P @ np.asarray(A, dtype=np.float64).T + np.asarray(b, dtype=np.float64)
    return np.ascontiguousarray(U, dtype=np.float32)


def rotation_field(n, origin, h, omega: float, center) -> np.ndarray:
    """Solid-body rotation about the z axis through ``center``."""
    A = np.array([[0.0, -omega, 0.0], [omega, 0.0, 0.0], [0.0, 0.0, 0.0]])
    c = np.asarray(center, dtype=np.float64)
    return affine_field(n, origin, h, A, -A @ c)


@dataclass
class FourierModes:
    k: np.ndarray       # (M, 3) wave vectors, units of the unit domain
    amp: np.ndarray     # (M,)
    e: np.ndarray       # (M, 3) unit polarisation, perpendicular to k
    phase: np.ndarray   # (M,)
    drift: np.ndarray   # (M,) per-cycle phase drift
    scale: float = 1.0

    @property
    def m(self) -> int:
        return int(self.k.shape[0])


def fourier_modes(seed: int, m: int = 64, kmin: float = 1.0, kmax: float = 16.0,
                  drift_max: float = 0.05, normalise: bool = True) -> FourierModes:
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    kmag = rng.uniform(kmin, kmax, size=m)
    k = d * kmag[:, None]
    # orthonormal pair perpendicular to k
    ref = np.where(np.abs(d[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    u1 = np.cross(d, ref)
    u1 /= np.linalg.norm(u1, axis=1, keepdims=True)
    u2 = np.cross(d, u1)
    ang = rng.uniform(0.0, 2.0 * np.pi, size=m)
    e = np.cos(ang)[:, None] * u1 + np.sin(ang)[:, None] * u2
    phase = rng.uniform(0.0, 2.0 * np.pi, size=m)
    drift = rng.uniform(0.0, drift_max, size=m)
    modes = FourierModes(k=k, amp=kmag ** (-5.0 / 6.0), e=e, phase=phase, drift=drift)
    if normalise:
        g = np.linspace(0.0, 1.0, 65)
        u = _fourier_eval(modes, g, g, g, 0)
        modes.scale = float(1.0 / np.sqrt(np.max(np.sum(u * u, axis=-1))))
    return modes


def _fourier_eval(modes: FourierModes, x, y, z, cycle: int) -> np.ndarray:
    """float64 (len z, len y, len x, 3) evaluation of the Fourier sum."""
    tw = 2.0 * np.pi
    X = np.exp(1j * tw * np.outer(x, modes.k[:, 0]))      # (nx, M)
    Y = np.exp(1j * tw * np.outer(y, modes.k[:, 1]))      # (ny, M)
    Zs = np.exp(1j * tw * np.outer(z, modes.k[:, 2]))     # (nz, M)
    W = modes.scale * modes.amp * np.exp(1j * (modes.phase + cycle * modes.drift))  # (M,)
    T = (Zs[:, None, :] * Y[None, :, :]).reshape(-1, modes.m)   # (nz*ny, M)
    out = np.empty((len(z), len(y), len(x), 3), dtype=np.float64)
    Tr, Ti = T.real.copy(), T.imag.copy()
    for comp in range(3):
        G = (W * modes.e[:, comp])[:, None] * X.T            # (M, nx)
        out[..., comp] = (Tr @ G.real - Ti @ G.imag).reshape(len(z), len(y), len(x))
    return out


def fourier_field(modes: FourierModes, n, origin, h, cycle: int) -> np.ndarray:
    """Fourier-mode turbulence at ``cycle`` on a block's nodes (float32)."""
    x, y, z = node_coords(n, origin, h)
    return np.ascontiguousarray(_fourier_eval(modes, x, y, z, cycle), dtype=np.float32)


def fourier_field_torch(modes: FourierModes, n, origin, h, cycle: int, device, dtype=None):
    """Same field as :func:`fourier_field`, evaluated with torch on ``device``
    in float64 and rounded to float32. Used to synthesise large inputs
    directly in device memory (the stand-in for the simulation).

    ``dtype=torch.float32`` evaluates the sum in single precision instead (a
    field within ~1e-5 relative of the float64 one, about 30x faster on the
    GPU): the per-cycle generator of the large in situ emulation."""
    import torch
    ft = torch.float64 if dtype is None else dtype
    x, y, z = (torch.as_tensor(v, dtype=torch.float64, device=device).to(ft)
               for v in node_coords(n, origin, h))
    k = torch.as_tensor(modes.k, dtype=torch.float64, device=device).to(ft)
    tw = 2.0 * np.pi
    X = torch.polar(torch.ones(len(x), modes.m, dtype=ft, device=device),
                    tw * torch.outer(x, k[:, 0]))
    Y = torch.polar(torch.ones(len(y), modes.m, dtype=ft, device=device),
                    tw * torch.outer(y, k[:, 1]))
    Zs = torch.polar(torch.ones(len(z), modes.m, dtype=ft, device=device),
                     tw * torch.outer(z, k[:, 2]))
    ph = torch.as_tensor(modes.phase + cycle * modes.drift, dtype=torch.float64, device=device).to(ft)
    amp = torch.as_tensor(modes.scale * modes.amp, dtype=torch.float64, device=device).to(ft)
    W = torch.polar(amp, ph)
    T = (Zs[:, None, :] * Y[None, :, :]).reshape(-1, modes.m)
    Tr, Ti = T.real.contiguous(), T.imag.contiguous()
    e = torch.as_tensor(modes.e, dtype=torch.float64, device=device).to(ft)
    out = torch.empty((len(z), len(y), len(x), 3), dtype=torch.float32, device=device)
    for comp in range(3):
        G = (W * e[:, comp])[:, None] * X.T
        out[..., comp] = (Tr @ G.real.contiguous() - Ti @ G.imag.contiguous()).reshape(
            len(z), len(y), len(x)).to(torch.float32)
    return out


def max_speed(field: np.ndarray) -> float:
    f = np.asarray(field, dtype=np.float64).reshape(-1, 3)
    return float(np.sqrt(np.max(np.sum(f * f, axis=1))))
