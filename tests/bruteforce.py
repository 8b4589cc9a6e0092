"""Brute-force references for pinning the oracle on tiny lattices.

These do not share the oracle's structure: the transition operator is built
as a dense matrix by scattering every source site's moves (Sec. 2.1: six
equally likely attempts, Metropolis acceptance of Eq. 1, rejection towards
solids and across non-periodic faces, jump factor alpha of Eq. 7), and
displacement statistics are taken from the full distribution over
(site, accumulated displacement) instead of from propagated moments.
"""
from __future__ import annotations

import math

import numpy as np

OFFSETS = ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))


def _target(x, y, z, off, shape, periodic):
    nz, ny, nx = shape
    c = [x + off[0], y + off[1], z + off[2]]
    n = [nx, ny, nz]
    for a in range(3):
        if not 0 <= c[a] < n[a]:
            if not periodic[a]:
                return None
            c[a] %= n[a]
    return (c[2] * ny + c[1]) * nx + c[0]


def moves(F, solid, periodic, alpha, kT=1.0, link_alpha=None):
    """List of (source, target, probability, offset) for every accepted move.

    link_alpha: optional symmetric function (i, j) -> alpha of the link between
    sites i and j (position-dependent diffusivity); alpha otherwise."""
    nz, ny, nx = F.shape
    Ff = F.reshape(-1)
    sf = solid.reshape(-1)
    out = []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = (z * ny + y) * nx + x
                if sf[i]:
                    continue
                for off in OFFSETS:
                    j = _target(x, y, z, off, F.shape, periodic)
                    if j is None or sf[j]:
                        continue
                    dE = (Ff[j] - Ff[i]) / kT
                    acc = math.exp(-dE) if dE > 0 else 1.0
                    a_ij = alpha if link_alpha is None else link_alpha(i, j)
                    out.append((i, j, a_ij / 6.0 * acc, off))
    return out


def transition_matrix(F, solid, periodic, alpha, kT=1.0, link_alpha=None):
    """Column-stochastic T with T[j, i] = P(i -> j) for one step (stay on the diagonal)."""
    N = F.size
    T = np.zeros((N, N))
    for i, j, p, _ in moves(F, solid, periodic, alpha, kT, link_alpha):
        T[j, i] += p
        T[i, i] -= p
    T[np.diag_indices(N)] += 1.0
    return T


def displacement_operator(F, solid, periodic, alpha, axis, kT=1.0):
    """D[j, i] = sum over moves i -> j of P(i -> j) * (displacement along axis)."""
    N = F.size
    D = np.zeros((N, N))
    for i, j, p, off in moves(F, solid, periodic, alpha, kT):
        D[j, i] += p * off[axis]
    return D


def distribution_msd(F, solid, periodic, alpha, rho0, nsteps, kT=1.0):
    """Exact MSD along each axis from the full (site, displacement) distribution.

    Returns (msd[3][nsteps+1], rho_n[nsteps+1][N]).  The accumulated
    displacement is the unwrapped path displacement.
    """
    N = F.size
    mv = {}
    stay = np.ones(N)
    for i, j, p, off in moves(F, solid, periodic, alpha, kT):
        mv.setdefault(i, []).append((j, p, off))
        stay[i] -= p
    r0 = np.asarray(rho0, dtype=np.float64).reshape(-1)
    P0 = r0.sum()
    dist = {(i, 0, 0, 0): r0[i] for i in range(N) if r0[i] != 0.0}
    msd = np.zeros((3, nsteps + 1))
    rhos = [r0.copy()]
    for n in range(1, nsteps + 1):
        nd = {}
        for (i, dx, dy, dz), p in dist.items():
            key = (i, dx, dy, dz)
            nd[key] = nd.get(key, 0.0) + p * stay[i]
            for j, q, off in mv.get(i, ()):
                key = (j, dx + off[0], dy + off[1], dz + off[2])
                nd[key] = nd.get(key, 0.0) + p * q
        dist = nd
        rho = np.zeros(N)
        acc = np.zeros(3)
        for (i, dx, dy, dz), p in dist.items():
            rho[i] += p
            acc += p * np.array([dx * dx, dy * dy, dz * dz], dtype=np.float64)
        msd[:, n] = acc / P0
        rhos.append(rho)
    return msd, rhos


def pore_clusters(solid, periodic):
    """Connected components of pore sites (6-neighbour, periodic where set)."""
    nz, ny, nx = solid.shape
    sf = solid.reshape(-1)
    label = -np.ones(sf.size, dtype=np.int64)
    cur = 0
    for start in range(sf.size):
        if sf[start] or label[start] >= 0:
            continue
        stack = [start]
        label[start] = cur
        while stack:
            i = stack.pop()
            z, rem = divmod(i, nx * ny)
            y, x = divmod(rem, nx)
            for off in OFFSETS:
                j = _target(x, y, z, off, solid.shape, periodic)
                if j is None or sf[j] or label[j] >= 0:
                    continue
                label[j] = cur
                stack.append(j)
        cur += 1
    return label.reshape(solid.shape), cur


def bits_round(v, drop):
    """Round doubles to nearest-even after dropping ``drop`` low significand bits.

    Integer manipulation of the IEEE-754 binary64 bit pattern (drop = 29 gives
    binary32 precision, drop = 45 gives bfloat16 precision), for finite
    positive normal values.
    """
    b = np.asarray(v, dtype=np.float64).view(np.int64).copy()
    lsb = (b >> drop) & 1
    b += ((np.int64(1) << (drop - 1)) - 1) + lsb
    b &= ~((np.int64(1) << drop) - 1)
    return b.view(np.float64)


def reservoir_operators(F, solid, periodic, alpha, reservoirs, kT=1.0):
    """One-step affine operator of a lattice with reservoir faces.

    A reservoir is a layer of fixed virtual sites just outside a face (face
    f = 2 a + side; side 0 lies below coordinate 0, side 1 above n_a - 1),
    given as (F_res, rho_res, m_res).  Every move that leaves the domain
    through a reservoir face is accepted by the Metropolis rule against F_res;
    every move from the reservoir into a boundary pore site against the
    site's F.  Returns dict with
      T      [N, N]  T[j, i] = P(i -> j) inside the domain, stay on the diagonal
                     (moves into a reservoir leave the domain);
      Win    [N, 6]  Win[i, f] = P(reservoir site of f -> i) per unit reservoir population;
      dface  [6, 3]  displacement of a move from face f into the domain;
      u, q   [3, N]  sum over all moves from i (reservoirs included) of p d_a and p d_a^2;
      Dax    [3][N, N] displacement operators of the moves inside the domain.
    """
    nz, ny, nx = F.shape
    N = F.size
    Ff = F.reshape(-1)
    sf = solid.reshape(-1)
    n = (nx, ny, nz)
    T = np.zeros((N, N))
    Win = np.zeros((N, 6))
    u = np.zeros((3, N))
    q = np.zeros((3, N))
    Dax = [np.zeros((N, N)) for _ in range(3)]
    dface = np.zeros((6, 3))
    for f in range(6):
        dface[f, f // 2] = 1.0 if f % 2 == 0 else -1.0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = (z * ny + y) * nx + x
                if sf[i]:
                    continue
                c = (x, y, z)
                for off in OFFSETS:
                    a = next(k for k in range(3) if off[k] != 0)
                    t = c[a] + off[a]
                    if 0 <= t < n[a] or periodic[a]:
                        j = _target(x, y, z, off, F.shape, periodic)
                        if sf[j]:
                            continue
                        dE = (Ff[j] - Ff[i]) / kT
                        p = alpha / 6.0 * (math.exp(-dE) if dE > 0 else 1.0)
                        T[j, i] += p
                        T[i, i] -= p
                        Dax[a][j, i] += p * off[a]
                    else:
                        f = 2 * a + (1 if off[a] > 0 else 0)
                        if reservoirs[f] is None:
                            continue
                        F_res = reservoirs[f][0]
                        dE = (F_res - Ff[i]) / kT
                        p = alpha / 6.0 * (math.exp(-dE) if dE > 0 else 1.0)
                        T[i, i] -= p
                        dE_in = (Ff[i] - F_res) / kT
                        Win[i, f] += alpha / 6.0 * (math.exp(-dE_in) if dE_in > 0 else 1.0)
                    u[a, i] += p * off[a]
                    q[a, i] += p * off[a] ** 2
    T[np.diag_indices(N)] += 1.0
    return dict(T=T, Win=Win, dface=dface, u=u, q=q, Dax=Dax)
