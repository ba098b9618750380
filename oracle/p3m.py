"""Reference P3M electrostatics for the periodic pipe -- test infrastructure.

This module is part of the oracle: only tests/, __graft_entry__.smoke() and
bench.py's CPU baseline may use it.  It shares no code with the CUDA library.

The paper computes the electrostatic force with P3M (App. A.2, Hockney and
Eastwood's particle-particle particle-mesh method; its extension to the
non-periodic pipe is cited, not printed).  Readings taken here: the pipe is
periodic along z with period L and isolated across (no images through the
wall); the Coulomb sum of particle i is

    s_i = sum_j sum_k q_j d / max(|d|, d_c)^3,   d = x_i - x_j - k L e_z,

which oracle.coulomb_periodic evaluates directly.  P3M splits the kernel
d / r^3 with an Ewald-type Gaussian screening of width 1/alpha:

    long range  K_L(d) = d [erf(alpha r) / r^3 - 2 alpha / sqrt(pi) exp(-alpha^2 r^2) / r^2],
    short range d / max(r, d_c)^3 - K_L(d), negligible beyond r_c (erfc(alpha r_c) small).

Steps, in order: (1) the long-range kernel summed over the periodic images
is sampled at the node offsets of a mesh that is periodic in z and, across,
twice as wide as the charge region so that the circular convolution of the
FFT equals the open one (Hockney's doubling); (2) charges are assigned to the
mesh with the triangular-shaped-cloud (TSC) weights; (3) the mesh sums are the
FFT convolution of charges and kernel, the kernel's transform divided by the
square of the TSC window's transform (sinc^3 per axis), which undoes the
smoothing that assignment and interpolation add; (4) the sums are
interpolated back with the same TSC weights (no self-force: the kernel is
odd); (5) the short-range part is summed directly over pairs closer than r_c
(minimum image along z).
Plain numpy, FP64, no blocking beyond what the steps state.
"""
import math

import numpy as np
from scipy.special import erf


class Desc:
    """Mesh and splitting parameters (wall units).

    M cells of width h = 2R/M across the diameter (nodes from -R - 2h, M + 5 of
    them, so that TSC stencils of particles inside the pipe stay on the mesh),
    Nz nodes along the period L, screening alpha, cut-off r_c, n_img images of
    the kernel each way before the far-field tail.
    """

    def __init__(self, R, L, M, Nz, alpha, rc, n_img=200):
        self.R, self.L, self.M, self.Nz = float(R), float(L), int(M), int(Nz)
        self.alpha, self.rc, self.n_img = float(alpha), float(rc), int(n_img)
        self.h = 2.0 * self.R / self.M
        self.hz = self.L / self.Nz
        self.Mx = self.M + 5
        self.x0 = -self.R - 2.0 * self.h
        self.Nx = 2 * self.Mx


def kernel_long(dx, dy, dz, alpha):
    """K_L(d) componentwise; near r = 0 (alpha r < 0.05, where the closed form cancels) its Taylor
    series 4 alpha^3 / (3 sqrt(pi)) d (1 - 3/5 (alpha r)^2 + 3/14 (alpha r)^4)."""
    r2 = dx * dx + dy * dy + dz * dz
    r = np.sqrt(r2)
    ar = alpha * r
    small = ar < 0.05
    with np.errstate(divide="ignore", invalid="ignore"):
        f = erf(ar) / (r2 * r) - 2.0 * alpha / math.sqrt(math.pi) * np.exp(-ar * ar) / r2
    u = ar * ar
    fs = 4.0 * alpha ** 3 / (3.0 * math.sqrt(math.pi)) * (1.0 - 0.6 * u + (3.0 / 14.0) * u * u)
    f = np.where(small, fs, f)
    return f * dx, f * dy, f * dz


def mesh_kernel(desc):
    """Long-range kernel summed over the z images, at every node offset: [3, Nx, Nx, Nz]."""
    N, Nz, h, hz, L = desc.Nx, desc.Nz, desc.h, desc.hz, desc.L
    off = np.arange(N)
    off = np.where(off > N // 2, off - N, off) * h
    offz = np.arange(Nz)
    offz = np.where(offz > Nz // 2, offz - Nz, offz) * hz      # z offsets in (-L/2, L/2]: symmetric image sums
    dx, dy, dz = np.meshgrid(off, off, offz, indexing="ij")
    G = np.zeros((3, N, N, Nz))
    for k in range(-desc.n_img, desc.n_img + 1):
        kx, ky, kz = kernel_long(dx, dy, dz - k * L, desc.alpha)
        G[0] += kx
        G[1] += ky
        G[2] += kz
    K = desc.n_img
    tail = 1.0 / (2.0 * (K + 0.5) ** 2) / L ** 3    # images beyond K in their far-field (1/r^2) form
    G[0] += 2.0 * dx * tail
    G[1] += 2.0 * dy * tail
    G[2] += -4.0 * dz * tail
    # the offset N/2 across is outside any pair of the charge region; it is left empty so that the
    # sampled kernel stays exactly odd (no self-force, no net force) under the FFT
    G[:, N // 2, :, :] = 0.0
    G[:, :, N // 2, :] = 0.0
    if Nz % 2 == 0:
        G[2, :, :, Nz // 2] = 0.0      # half a period along z: the periodic sum of the odd z-component vanishes
    return G


def influence(desc, G=None):
    """Transforms of the three kernel components divided by the squared TSC window: [3, Nx, Nx, Nz//2+1]."""
    G = mesh_kernel(desc) if G is None else G
    wx = np.sinc(np.fft.fftfreq(desc.Nx)) ** 6          # (sinc^3)^2 along x and y
    wz = np.sinc(np.fft.rfftfreq(desc.Nz)) ** 6
    W = wx[:, None, None] * wx[None, :, None] * wz[None, None, :]
    return np.stack([np.fft.rfftn(G[c], axes=(0, 1, 2)) / W for c in range(3)])


def _tsc(t):
    """Nearest node and the three TSC weights for a coordinate in node units."""
    i0 = np.rint(t).astype(np.int64)
    d = t - i0
    return i0, np.stack([0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2], -1)


def _stencil(desc, x, y, z):
    ix, wx = _tsc((x - desc.x0) / desc.h)
    iy, wy = _tsc((y - desc.x0) / desc.h)
    iz, wz = _tsc(z / desc.hz)
    return ix, wx, iy, wy, iz, wz


def assign(desc, x, y, z, q):
    Q = np.zeros((desc.Nx, desc.Nx, desc.Nz))
    ix, wx, iy, wy, iz, wz = _stencil(desc, x, y, z)
    for a in range(3):
        for b in range(3):
            for c in range(3):
                np.add.at(Q, (ix + a - 1, iy + b - 1, (iz + c - 1) % desc.Nz), q * wx[:, a] * wy[:, b] * wz[:, c])
    return Q


def interpolate(desc, A, x, y, z):
    ix, wx, iy, wy, iz, wz = _stencil(desc, x, y, z)
    out = np.zeros(len(x))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                out += A[ix + a - 1, iy + b - 1, (iz + c - 1) % desc.Nz] * wx[:, a] * wy[:, b] * wz[:, c]
    return out


def mesh_sums(desc, Gh, x, y, z, q):
    """Long-range Coulomb sums [n, 3] by assignment, FFT convolution with the influence
    function Gh (from influence()) and interpolation."""
    shape = (desc.Nx, desc.Nx, desc.Nz)
    Q = np.fft.rfftn(assign(desc, x, y, z, q), axes=(0, 1, 2))
    out = np.zeros((len(x), 3))
    for c in range(3):
        A = np.fft.irfftn(Q * Gh[c], s=shape, axes=(0, 1, 2))
        out[:, c] = interpolate(desc, A, x, y, z)
    return out


def pp_sums(desc, x, y, z, q, contact, alive=None):
    """Short-range sums: q_j (d / max(r, d_c)^3 - K_L(d)) over j != i with r < r_c."""
    n = len(x)
    alive = np.ones(n, bool) if alive is None else np.asarray(alive, bool)
    out = np.zeros((n, 3))
    for i in range(n):
        if not alive[i]:
            continue
        dx, dy, dz = x[i] - x, y[i] - y, z[i] - z
        dz = dz - desc.L * np.rint(dz / desc.L)
        r = np.sqrt(dx * dx + dy * dy + dz * dz)
        m = (r < desc.rc) & alive
        m[i] = False
        dx, dy, dz, r, qj = dx[m], dy[m], dz[m], r[m], q[m]
        rr = np.maximum(r, contact)
        lx, ly, lz = kernel_long(dx, dy, dz, desc.alpha)
        out[i, 0] = np.sum(qj * (dx / rr ** 3 - lx))
        out[i, 1] = np.sum(qj * (dy / rr ** 3 - ly))
        out[i, 2] = np.sum(qj * (dz / rr ** 3 - lz))
    return out


def coulomb_sums(desc, x, y, z, q, contact, Gh=None, alive=None):
    """P3M Coulomb sums [n, 3]; removed particles (alive = 0) neither feel nor exert forces."""
    alive = np.ones(len(x), bool) if alive is None else np.asarray(alive, bool)
    Gh = influence(desc) if Gh is None else Gh
    qa = np.where(alive, q, 0.0)
    s = mesh_sums(desc, Gh, x, y, z, qa) + pp_sums(desc, x, y, z, qa, contact, alive)
    s[~alive] = 0.0
    return s
