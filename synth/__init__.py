"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module holds problem *data* only: mesh node coordinates and time nodes,
seeded random numbers, the closed-form manufactured solutions of the model
problem and their right-hand sides, Gaussian wave packets, and the sizes of
the standard workloads.  It contains none of the discretisation or solver
arithmetic (no element matrices, no assembly, no eigen-decomposition, no
solves): the oracle and the CUDA path each implement those on their own.

Model problem (Section 1, eq. (1)):  i d/dt psi - Laplace_x psi = f  in
Omega x (0, T), psi = 0 on the boundary, psi(., 0) = psi0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "uniform_time_nodes", "graded_time_nodes", "interior_coords", "cn01",
    "PacketParams", "packet_params", "packet_values",
    "psi_c1", "f_c1", "psi0_c1", "psi_paper", "f_paper",
    "Problem", "config_problem", "batch_problems", "square_delaunay_mesh", "cube_tet_mesh",
    "packet_values_nd",
]


# ---------------------------------------------------------------- meshes
def uniform_time_nodes(N_t: int, T: float) -> np.ndarray:
    """Uniform temporal mesh t_l = T l / N_t, l = 0..N_t (Section 4, eq. Mesh_t)."""
    return T * np.arange(N_t + 1, dtype=np.float64) / N_t


def graded_time_nodes(T: float, q: float = 1.5, N0: int = 64, levels: int = 0) -> np.ndarray:
    """Graded temporal mesh t_l = T (l/N0)^q, l = 0..N0 (Section 4, Table 3),
    refined `levels` times by bisecting every element (uniform refinement)."""
    t = T * (np.arange(N0 + 1, dtype=np.float64) / N0) ** q
    for _ in range(levels):
        mid = 0.5 * (t[:-1] + t[1:])
        out = np.empty(2 * len(t) - 1)
        out[0::2] = t
        out[1::2] = mid
        t = out
    return t


def interior_coords(n: int, Lx: float = 1.0, Ly: float = 1.0):
    """Coordinates of the (n-1)^2 interior nodes of the n x n-square grid of
    (0,Lx) x (0,Ly), lexicographic with x1 fastest.  Returns (x1, x2)."""
    m = n - 1
    i = np.arange(1, n, dtype=np.float64)
    x1 = np.tile(i * (Lx / n), m)
    x2 = np.repeat(i * (Ly / n), m)
    return x1, x2


def square_delaunay_mesh(n: int, jitter: float = 0.3, seed: int = 0, L: float = 1.0):
    """An unstructured triangulation of (0,L)^2: the Delaunay triangulation of the (n+1)^2 grid
    points with every interior point moved by up to `jitter` h in each coordinate (h = L/n,
    seeded), boundary points fixed.  Returns (coords[V, 2], triangles[C, 3]) with
    counter-clockwise triangles."""
    from scipy.spatial import Delaunay

    rng = np.random.Generator(np.random.PCG64(seed))
    h = L / n
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    xy = np.stack([i.ravel() * h, j.ravel() * h], axis=1)
    inner = (i.ravel() > 0) & (i.ravel() < n) & (j.ravel() > 0) & (j.ravel() < n)
    xy[inner] += rng.uniform(-jitter * h, jitter * h, size=(int(inner.sum()), 2))
    tri = Delaunay(xy).simplices.astype(np.int64)
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    tri[cross < 0] = tri[cross < 0][:, [0, 2, 1]]
    return xy, tri


def cube_tet_mesh(n: int, jitter: float = 0.2, seed: int = 0, L: float = 1.0):
    """A tetrahedral mesh of (0,L)^3: n^3 cubes, each split into the 6 tetrahedra around its main
    diagonal (a conforming split), interior vertices moved by up to `jitter` h in each coordinate
    (seeded).  Returns (coords[V, 3], tets[C, 4])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = L / n
    g = np.arange(n + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    idx = lambda a, b, c: (a * (n + 1) + b) * (n + 1) + c   # noqa: E731
    xyz = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1).astype(np.float64) * h
    inner = np.all((np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1) > 0) &
                   (np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1) < n), axis=1)
    xyz[inner] += rng.uniform(-jitter * h, jitter * h, size=(int(inner.sum()), 3))
    c0 = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), axis=-1).reshape(-1, 3)
    # the 6 monotone lattice paths from corner (0,0,0) to (1,1,1)
    paths = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tets = []
    for pth in paths:
        v = [c0.copy()]
        cur = c0.copy()
        for ax in pth:
            cur = cur.copy()
            cur[:, ax] += 1
            v.append(cur)
        tets.append(np.stack([idx(q[:, 0], q[:, 1], q[:, 2]) for q in v], axis=1))
    return xyz, np.concatenate(tets, axis=0).astype(np.int64)


def packet_values_nd(p: "PacketParams", x: np.ndarray) -> np.ndarray:
    """Gaussian packets at points x (P, d), d = 2 or 3: the parameters' centres and momenta give
    the first two components; a third coordinate is centred at 0.5 with zero momentum."""
    d = x.shape[1]
    out = np.zeros(x.shape[0], dtype=np.complex128)
    for s, c, k in zip(p.sigma, p.centre, p.k):
        cc = np.full(d, 0.5)
        kk = np.zeros(d)
        cc[:2] = c[:2]
        kk[:2] = k[:2]
        r2 = ((x - cc) ** 2).sum(axis=1)
        out += np.exp(-r2 / (2 * s * s)) * np.exp(1j * (x @ kk))
    return out


# ---------------------------------------------------------------- random
def cn01(shape, seed: int) -> np.ndarray:
    """Seeded standard complex normal CN(0,1) = (N(0,1) + i N(0,1)) / sqrt(2), PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) / math.sqrt(2.0)


@dataclass
class PacketParams:
    sigma: np.ndarray   # (P,)
    centre: np.ndarray  # (P, 2)
    k: np.ndarray       # (P, 2)


def packet_params(seed: int, count: int = 4, sigma=(0.05, 0.1), centre=(0.3, 0.7),
                  kmax: float = 20.0) -> PacketParams:
    """Seeded parameters of `count` Gaussian wave packets: sigma ~ U(sigma),
    centre ~ U(centre)^2, momentum k ~ U(-kmax, kmax)^2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = rng.uniform(sigma[0], sigma[1], size=count)
    c = rng.uniform(centre[0], centre[1], size=(count, 2))
    k = rng.uniform(-kmax, kmax, size=(count, 2))
    return PacketParams(s, c, k)


def packet_values(p: PacketParams, x1: np.ndarray, x2: np.ndarray) -> np.ndarray:
    """Sum of unnormalised Gaussian packets exp(-|x-c|^2/(2 sigma^2)) e^{i k.x}."""
    out = np.zeros(np.broadcast(x1, x2).shape, dtype=np.complex128)
    for s, c, k in zip(p.sigma, p.centre, p.k):
        r2 = (x1 - c[0]) ** 2 + (x2 - c[1]) ** 2
        out += np.exp(-r2 / (2.0 * s * s)) * np.exp(1j * (k[0] * x1 + k[1] * x2))
    return out


# ---------------------------------------------------------------- manufactured solutions
def psi_c1(x1, x2, t):
    """psi = sin(pi x1) sin(pi x2) (1 + t) e^{-i t}."""
    return np.sin(np.pi * x1) * np.sin(np.pi * x2) * (1.0 + t) * np.exp(-1j * t)


def f_c1(x1, x2, t):
    """f = i d/dt psi - Laplace psi for psi_c1:  S(x) e^{-it} [(1 + 2 pi^2)(1 + t) + i]."""
    S = np.sin(np.pi * x1) * np.sin(np.pi * x2)
    return S * np.exp(-1j * t) * ((1.0 + 2.0 * np.pi ** 2) * (1.0 + t) + 1j)


def psi0_c1(x1, x2):
    return np.sin(np.pi * x1) * np.sin(np.pi * x2) + 0j


def psi_paper(x1, x2, t):
    """Exact solution of Section 4: e^{it} sin(pi x1) sin(pi x2) sin(t x1 x2); psi0 = 0."""
    return np.exp(1j * t) * np.sin(np.pi * x1) * np.sin(np.pi * x2) * np.sin(t * x1 * x2)


def f_paper(x1, x2, t):
    """f = i d/dt psi - Laplace psi for psi_paper (a = sin pi x1, b = sin pi x2, c = sin(t x1 x2))."""
    a = np.sin(np.pi * x1)
    b = np.sin(np.pi * x2)
    ca = np.cos(np.pi * x1)
    cb = np.cos(np.pi * x2)
    arg = t * x1 * x2
    c = np.sin(arg)
    cc = np.cos(arg)
    e = np.exp(1j * t)
    dt = 1j * e * a * b * c + e * a * b * x1 * x2 * cc
    lap = (-(2.0 * np.pi ** 2 + t * t * (x1 * x1 + x2 * x2)) * a * b * c
           + 2.0 * np.pi * t * cc * (x2 * ca * b + x1 * a * cb))
    return 1j * dt - e * lap


# ---------------------------------------------------------------- workloads
@dataclass
class Problem:
    """One space-time problem: n x n squares on (0,Lx)x(0,Ly), time degree p_t on nodes t."""
    n: int
    p_t: int
    t_nodes: np.ndarray
    Lx: float = 1.0
    Ly: float = 1.0
    name: str = ""
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.n - 1

    @property
    def n_x(self) -> int:
        return (self.n - 1) ** 2

    @property
    def n_t(self) -> int:
        return self.p_t * (len(self.t_nodes) - 1)

    @property
    def unknowns(self) -> int:
        return self.n_x * self.n_t


def config_problem(name: str) -> Problem:
    """The standard workloads by name.

    c1        16x16 squares, P1 time, 16 uniform elements, T=1 (3,600 unknowns)
    c2        256x256 squares, P1 time, 512 uniform elements, T=1 (33,292,800)
    c2check   64x64 squares, P1 time, 128 uniform elements, T=1 (508,032)
    c3        384x384 squares, P2 time, 512 uniform elements, T=2 (150,209,536)
    c4        128x128 squares, P1 time, 256 uniform elements, T=1 (4,129,024)
    c2small   256x256 squares, P1 time, 16 uniform elements, T=1/32 (profiling case)
    c3small   384x384 squares, P2 time, 8 uniform elements, T=1/32 (profiling case)
    paperJ    paper's level-J mesh: (32 2^J)^2 squares, P1, 64 2^J elements, T=5
    """
    if name == "c1":
        return Problem(16, 1, uniform_time_nodes(16, 1.0), name=name, seed=1)
    if name == "c2":
        return Problem(256, 1, uniform_time_nodes(512, 1.0), name=name, seed=2)
    if name == "c2check":
        return Problem(64, 1, uniform_time_nodes(128, 1.0), name=name, seed=2)
    if name == "c3":
        return Problem(384, 2, uniform_time_nodes(512, 2.0), name=name, seed=3)
    if name == "c4":
        return Problem(128, 1, uniform_time_nodes(256, 1.0), name=name, seed=4)
    if name == "c3small":
        # the 384x384 spatial band of c3 with P2 time on 8 elements (n_t = 16): a small case for profiling
        return Problem(384, 2, uniform_time_nodes(8, 2.0 / 64), name=name, seed=3)
    if name == "c2small":
        # the 256x256 spatial band of c2 with 16 time elements: a small case for profiling
        return Problem(256, 1, uniform_time_nodes(16, 1.0 / 32), name=name, seed=2)
    if name.startswith("paperJ"):
        J = int(name[6:])
        return Problem(32 * 2 ** J, 1, uniform_time_nodes(64 * 2 ** J, 5.0), name=name, seed=0)
    raise KeyError(name)


def batch_problems(count: int = 64, seed: int = 5, n_choices=None, Nt_range=(32, 512),
                   T_range=(0.5, 2.0)) -> list:
    """Seeded batch of uneven problems: n ~ U{32,48,...,192}, p_t ~ U{1,2},
    N_t ~ U{Nt_range}, T ~ U(T_range); each carries its own packet/forcing seed."""
    if n_choices is None:
        n_choices = list(range(32, 193, 16))
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(rng.choice(n_choices))
        p_t = int(rng.integers(1, 3))
        N_t = int(rng.integers(Nt_range[0], Nt_range[1] + 1))
        T = float(rng.uniform(*T_range))
        forced = bool(rng.integers(0, 2))
        fk = (int(rng.integers(1, 4)), int(rng.integers(1, 4)))
        omega = float(rng.uniform(0.0, 10.0))
        c = complex(*(rng.standard_normal(2) / math.sqrt(2.0)))
        out.append(Problem(n, p_t, uniform_time_nodes(N_t, T), name=f"b{i}", seed=seed * 1000 + i,
                           extra=dict(forced=forced, fk=fk, omega=omega, c=c)))
    return out


def dof_times(p_t: int, t_nodes) -> np.ndarray:
    """Times of the temporal DOFs including t_0: the mesh nodes (P1), nodes and midpoints (P2)."""
    t = np.asarray(t_nodes, dtype=np.float64)
    if p_t == 1:
        return t.copy()
    tf = np.empty(2 * len(t) - 1)
    tf[0::2] = t
    tf[1::2] = 0.5 * (t[:-1] + t[1:])
    return tf


def batch_inputs(pr: Problem):
    """Inputs of one problem of the uneven batch: psi0 = its seeded 4-packet sum at the interior
    nodes, and the forcing f = c sin(k1 pi x1) sin(k2 pi x2) e^{i omega t} (or f = 0) in separable
    form f(x, t) = a(t) b(x): returns (psi0 (n_x,), a at the DOF times incl. t_0, b (n_x,)), with
    a = b = None for an unforced problem."""
    x1, x2 = interior_coords(pr.n, pr.Lx, pr.Ly)
    psi0 = packet_values(packet_params(pr.seed), x1, x2)
    e = pr.extra or {}
    if not e.get("forced", False):
        return psi0, None, None
    k1, k2 = e["fk"]
    a = complex(e["c"]) * np.exp(1j * e["omega"] * dof_times(pr.p_t, pr.t_nodes))
    b = (np.sin(k1 * np.pi * x1) * np.sin(k2 * np.pi * x2)).astype(np.complex128)
    return psi0, a, b


def psi_c1_derivs(x1, x2, t):
    """(d_t, d_x1, d_x2) of psi_c1."""
    a, b = np.sin(np.pi * x1), np.sin(np.pi * x2)
    g = (1.0 + t) * np.exp(-1j * t)
    gt = np.exp(-1j * t) * (1.0 - 1j * (1.0 + t))
    return (a * b * gt, np.pi * np.cos(np.pi * x1) * b * g, np.pi * a * np.cos(np.pi * x2) * g)


def psi_paper_derivs(x1, x2, t):
    """(d_t, d_x1, d_x2) of psi_paper."""
    a, b = np.sin(np.pi * x1), np.sin(np.pi * x2)
    arg = t * x1 * x2
    c, cc = np.sin(arg), np.cos(arg)
    e = np.exp(1j * t)
    d_t = 1j * e * a * b * c + e * a * b * x1 * x2 * cc
    d_x1 = e * b * (np.pi * np.cos(np.pi * x1) * c + a * t * x2 * cc)
    d_x2 = e * a * (np.pi * np.cos(np.pi * x2) * c + b * t * x1 * cc)
    return d_t, d_x1, d_x2
