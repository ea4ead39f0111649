"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds none of the solver's arithmetic: it only draws random
numbers and turns them into the inputs the solver is run on.

* SU(3) gauge links  U_mu(n) = exp(i * eps * X),  X = sum_a xi_a lambda_a / 2,
  xi_a ~ N(0,1) (lambda_a the Gell-Mann matrices), exponential by a Taylor
  series to order 20 in FP64, then re-unitarised (Gram-Schmidt on rows 1-2,
  row 3 = conj(row1 x row2), so det U = 1).
* Gaussian spinor sources: real and imaginary parts iid N(0,1).
* Point sources: b = delta(n,0) delta(alpha,alpha0) delta(a,a0).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: output i is mix(seed + (i+1) * 0x9E3779B97F4A7C15). Uniforms in
(0,1) take the top 53 bits plus one half ulp; normals come from Box-Muller
(normal 2k uses cos, normal 2k+1 uses sin of the same uniform pair).

Layouts (canonical, shared by every caller):
  site n = x + Lx*(y + Ly*(z + Lz*t)), dims = (Lx, Ly, Lz, Lt)
  links   complex128 [V][4 mu][3][3]     (mu = 0..3 is x, y, z, t)
  spinor  complex128 [V][4 spin][3 colour]

Draw order for links: site-major, then mu, then xi_1..xi_8.

The numpy path is the reference path. ``gauge_field(..., device="cuda")``
runs the same steps with torch on a GPU (used only to create very large
fields quickly); the integer stream is identical, the transcendental
functions may differ in the last ulp.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of SplitMix64 seeded with ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start, start + count, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (i + np.uint64(1)) * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1)."""
    z = splitmix64(seed, start, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normals(seed: int, count: int) -> np.ndarray:
    """``count`` standard normals by Box-Muller over the uniform stream."""
    npair = (count + 1) // 2
    u = uniforms(seed, 0, 2 * npair).reshape(npair, 2)
    rad = np.sqrt(-2.0 * np.log(u[:, 0]))
    ang = 2.0 * math.pi * u[:, 1]
    out = np.empty((npair, 2))
    out[:, 0] = rad * np.cos(ang)
    out[:, 1] = rad * np.sin(ang)
    return out.reshape(-1)[:count]


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_1..lambda_8, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / math.sqrt(3)
    lam[7][2, 2] = -2 / math.sqrt(3)
    return lam


def volume(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


def _expm_taylor(A: np.ndarray, order: int = 20) -> np.ndarray:
    """exp(A) for a batch of 3x3 matrices by Horner evaluation of the Taylor series."""
    eye = np.broadcast_to(np.eye(3, dtype=A.dtype), A.shape)
    R = eye.copy()
    for k in range(order, 0, -1):
        R = eye + (A @ R) / k
    return R


def reunitarise(U: np.ndarray) -> np.ndarray:
    """Project a batch of near-SU(3) matrices back onto SU(3) (rows 1-2 Gram-Schmidt)."""
    r1 = U[..., 0, :]
    r2 = U[..., 1, :]
    r1 = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1, keepdims=True))
    r2 = r2 - np.sum(np.conj(r1) * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.sqrt(np.sum(np.abs(r2) ** 2, axis=-1, keepdims=True))
    r3 = np.conj(np.cross(r1, r2))
    return np.stack([r1, r2, r3], axis=-2)


def gauge_field(dims, eps: float = 0.3, seed: int = 1000, chunk_sites: int = 1 << 16,
                device: str = "cpu"):
    """Random SU(3) links U_mu(n) = exp(i eps X), complex128 array [V,4,3,3].

    With ``device`` other than "cpu" the result is a torch tensor on that device.
    """
    V = volume(dims)
    if device != "cpu":
        return _gauge_field_torch(dims, eps, seed, device)
    lam = gell_mann() / 2.0
    out = np.empty((V, 4, 3, 3), dtype=np.complex128)
    for s0 in range(0, V, chunk_sites):
        s1 = min(V, s0 + chunk_sites)
        # normals are drawn in global order; chunk boundaries fall on even offsets
        nstart = s0 * 32
        xi = _normals_range(seed, nstart, (s1 - s0) * 32).reshape(s1 - s0, 4, 8)
        X = np.einsum("nma,aij->nmij", xi, lam)
        out[s0:s1] = reunitarise(_expm_taylor(1j * eps * X))
    return out


def _normals_range(seed: int, start: int, count: int) -> np.ndarray:
    """Normals start .. start+count-1 of the stream (start and count even)."""
    assert start % 2 == 0 and count % 2 == 0
    u = uniforms(seed, start, count).reshape(-1, 2)
    rad = np.sqrt(-2.0 * np.log(u[:, 0]))
    ang = 2.0 * math.pi * u[:, 1]
    out = np.empty((u.shape[0], 2))
    out[:, 0] = rad * np.cos(ang)
    out[:, 1] = rad * np.sin(ang)
    return out.reshape(-1)


def gaussian_spinor(dims, seed: int = 2000, nrhs: int = 1) -> np.ndarray:
    """Gaussian complex source(s): complex128 [nrhs, V, 4, 3] (re, im iid N(0,1))."""
    V = volume(dims)
    n = normals(seed, 2 * 12 * V * nrhs).reshape(nrhs, V, 4, 3, 2)
    return n[..., 0] + 1j * n[..., 1]


def point_sources(dims) -> np.ndarray:
    """The 12 spin-colour point sources at the origin: complex128 [12, V, 4, 3]."""
    V = volume(dims)
    b = np.zeros((12, V, 4, 3), dtype=np.complex128)
    for k in range(12):
        b[k, 0, k // 3, k % 3] = 1.0
    return b


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """Random SU(3) matrices g(n), complex128 [V,3,3] (same recipe as a link, eps = 1)."""
    V = volume(dims)
    lam = gell_mann() / 2.0
    xi = normals(seed, V * 8).reshape(V, 8)
    X = np.einsum("na,aij->nij", xi, lam)
    return reunitarise(_expm_taylor(1j * 1.0 * X))


def unit_gauge(dims) -> np.ndarray:
    V = volume(dims)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1.0
    return U


# ---------------------------------------------------------------------------
# torch path for large fields (same integer stream, same steps)
# ---------------------------------------------------------------------------

def _to_i64(v: int) -> int:
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


def _srl(z, k):
    import torch
    return (z >> k) & ((1 << (64 - k)) - 1)


def _uniforms_torch(seed: int, start: int, count: int, device):
    import torch
    i = torch.arange(start, start + count, dtype=torch.int64, device=device)
    z = (i + 1) * _to_i64(_GOLDEN) + _to_i64(seed)
    z = (z ^ _srl(z, 30)) * _to_i64(_M1)
    z = (z ^ _srl(z, 27)) * _to_i64(_M2)
    z = z ^ _srl(z, 31)
    return (_srl(z, 11).to(torch.float64) + 0.5) * (1.0 / 9007199254740992.0)


def _gauge_field_torch(dims, eps, seed, device, chunk_sites: int = 1 << 20):
    import torch
    V = volume(dims)
    lam = torch.as_tensor(gell_mann() / 2.0, device=device)
    out = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device=device)
    eye = torch.eye(3, dtype=torch.complex128, device=device)
    for s0 in range(0, V, chunk_sites):
        s1 = min(V, s0 + chunk_sites)
        u = _uniforms_torch(seed, s0 * 32, (s1 - s0) * 32, device).view(-1, 2)
        rad = torch.sqrt(-2.0 * torch.log(u[:, 0]))
        ang = 2.0 * math.pi * u[:, 1]
        xi = torch.stack([rad * torch.cos(ang), rad * torch.sin(ang)], dim=1).reshape(s1 - s0, 4, 8)
        X = torch.einsum("nma,aij->nmij", xi.to(torch.complex128), lam)
        A = 1j * eps * X
        R = eye.expand_as(A).clone()
        for k in range(20, 0, -1):
            R = eye + (A @ R) / k
        r1, r2 = R[..., 0, :], R[..., 1, :]
        r1 = r1 / torch.sqrt((r1.abs() ** 2).sum(-1, keepdim=True))
        r2 = r2 - (r1.conj() * r2).sum(-1, keepdim=True) * r1
        r2 = r2 / torch.sqrt((r2.abs() ** 2).sum(-1, keepdim=True))
        r3 = torch.linalg.cross(r1, r2).conj()
        out[s0:s1] = torch.stack([r1, r2, r3], dim=-2)
    return out


def gaussian_spinor_torch(dims, seed: int, nrhs: int, device):
    """Same stream as :func:`gaussian_spinor`, created on ``device`` with torch."""
    import torch
    V = volume(dims)
    cnt = 2 * 12 * V * nrhs
    u = _uniforms_torch(seed, 0, cnt, device).view(-1, 2)
    rad = torch.sqrt(-2.0 * torch.log(u[:, 0]))
    ang = 2.0 * math.pi * u[:, 1]
    n = torch.stack([rad * torch.cos(ang), rad * torch.sin(ang)], dim=1).reshape(nrhs, V, 4, 3, 2)
    return torch.complex(n[..., 0], n[..., 1])
