"""Seeded synthetic inputs: convection-diffusion systems Ax = b.

This module only builds problem instances (matrix, right-hand side, random
coefficient field). It holds none of the solver's arithmetic: no splitting,
no iteration, no precision handling. Both the CUDA path and the CPU oracle
consume what it produces, so that they are compared on identical inputs.

Problem (paper §4.1, the 3D convection-diffusion experiment): centred
differences of  -div(k grad u) + beta * (u_x + u_y [+ u_z]) = f  on the unit
square/cube with homogeneous Dirichlet boundary conditions, on an N^dim grid
of interior nodes, h = 1/(N+1). Every row is multiplied by h^2, which is the
scaling the paper uses: for k = 1 and beta = 1 the matrix is the Kronecker sum
T_x (x) I (x) I + I (x) T_y (x) I + I (x) I (x) T_z with diagonal 6 and
off-diagonals -1 - r (lower) and -1 + r (upper), r = h/2.

With beta the convection coefficient becomes c = beta*h/2 per direction. With
a face coefficient k_f the row of node i is

    diag      = sum over its 2*dim faces of k_f
    lower nb  = -k_f - c      (neighbour at i - e_d)
    upper nb  = -k_f + c      (neighbour at i + e_d)

where a face on the boundary contributes to the diagonal only.

Node numbering is x fastest: i = ix + N*iy + N^2*iz. Columns in each CSR row
are ascending.

Face-coefficient layout (3D), one FP64 array per direction, C order:
    kx: shape (N, N, N+1)  index (iz, iy, fx), face fx between nodes fx-1 and fx
    ky: shape (N, N+1, N)  index (iz, fy, ix)
    kz: shape (N+1, N, N)  index (fz, iy, ix)
Face f along d sits at coordinate (f + 1/2) h; node j sits at (j + 1) h.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Csr", "Problem", "convdiff_csr", "grf_faces", "manufactured_solution",
    "rhs_from_solution", "make_problem", "random_vector",
]


@dataclasses.dataclass
class Csr:
    """Compressed sparse rows, int32 indices, FP64 values."""
    n: int
    row_ptr: np.ndarray   # int32, n+1
    col_idx: np.ndarray   # int32, nnz
    val: np.ndarray       # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col_idx, self.row_ptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        return self.to_scipy().toarray()


@dataclasses.dataclass
class Problem:
    """One synthetic instance: A, b, the exact discrete solution if known,
    and the structure needed by matrix-free kernels."""
    name: str
    dim: int
    N: int
    beta: float
    A: Csr
    b: np.ndarray
    x_exact: np.ndarray | None
    faces: tuple | None          # (kx, ky, kz) FP64 or None when k = 1

    @property
    def n(self) -> int:
        return self.A.n


def _face_shapes(N: int):
    return ((N, N, N + 1), (N, N + 1, N), (N + 1, N, N))


def convdiff_csr(dim: int, N: int, beta: float, faces=None) -> Csr:
    """Assemble the h^2-scaled centred-difference operator as CSR.

    dim: 2 or 3. faces: None (k = 1) or, for dim = 3, (kx, ky, kz) in the
    layout described in the module docstring.
    """
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    if N < 1:
        raise ValueError("N must be >= 1")
    if faces is not None and dim != 3:
        raise ValueError("face coefficients are supported for dim = 3 only")
    h = 1.0 / (N + 1)
    c = beta * h / 2.0
    n = N ** dim
    idx = np.arange(n, dtype=np.int64)
    coords = [(idx // (N ** d)) % N for d in range(dim)]   # d = 0 is x

    # k on the lower and upper face of every node, per direction
    k_lo, k_hi = [], []
    for d in range(dim):
        if faces is None:
            k_lo.append(np.ones(n))
            k_hi.append(np.ones(n))
            continue
        F = np.asarray(faces[d], dtype=np.float64)
        if F.shape != _face_shapes(N)[d]:
            raise ValueError(f"face array {d} has shape {F.shape}, want {_face_shapes(N)[d]}")
        ix, iy, iz = coords
        if d == 0:
            lo, hi = F[iz, iy, ix], F[iz, iy, ix + 1]
        elif d == 1:
            lo, hi = F[iz, iy, ix], F[iz, iy + 1, ix]
        else:
            lo, hi = F[iz, iy, ix], F[iz + 1, iy, ix]
        k_lo.append(lo)
        k_hi.append(hi)

    diag = np.zeros(n)
    for d in range(dim):
        diag += k_lo[d] + k_hi[d]

    # candidate entries in ascending column order: (-e_{dim-1}, ..., -e_0, 0, +e_0, ..., +e_{dim-1})
    cols, vals, masks = [], [], []
    for d in reversed(range(dim)):
        stride = N ** d
        cols.append(idx - stride)
        vals.append(-k_lo[d] - c)
        masks.append(coords[d] > 0)
    cols.append(idx)
    vals.append(diag)
    masks.append(np.ones(n, dtype=bool))
    for d in range(dim):
        stride = N ** d
        cols.append(idx + stride)
        vals.append(-k_hi[d] + c)
        masks.append(coords[d] < N - 1)
    C = np.stack(cols, axis=1)
    V = np.stack(vals, axis=1)
    Mk = np.stack(masks, axis=1)
    counts = Mk.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 index range")
    return Csr(n=n, row_ptr=row_ptr.astype(np.int32),
               col_idx=C[Mk].astype(np.int32), val=V[Mk].astype(np.float64))


def grf_faces(N: int, seed: int, sigma: float = 1.0, ell: float = 0.1,
              nfeat: int = 1024):
    """k = exp(g) on the cell faces of an N^3 grid, g a Gaussian random field.

    g has mean 0 and squared-exponential covariance sigma^2 exp(-|d|^2/(2 ell^2)),
    sampled by nfeat random Fourier features: g(x) = sigma sqrt(2/K) sum_j
    cos(w_j . x + phi_j), w_j ~ N(0, ell^-2 I), phi_j ~ U[0, 2 pi).
    Returns (kx, ky, kz) in the layout of the module docstring.
    """
    rng = np.random.default_rng(seed)
    W = rng.normal(0.0, 1.0 / ell, size=(nfeat, 3))
    phi = rng.uniform(0.0, 2.0 * math.pi, size=nfeat)
    amp = sigma * math.sqrt(2.0 / nfeat)
    h = 1.0 / (N + 1)
    nodes = (np.arange(N) + 1.0) * h
    facec = (np.arange(N + 1) + 0.5) * h

    def field(xs, ys, zs):
        Ex = np.exp(1j * np.outer(W[:, 0], xs))                       # (K, nx)
        Ey = np.exp(1j * np.outer(W[:, 1], ys))                       # (K, ny)
        Ez = np.exp(1j * (np.outer(W[:, 2], zs) + phi[:, None]))      # (K, nz)
        out = np.empty((len(zs), len(ys), len(xs)))
        for iz in range(len(zs)):
            out[iz] = ((Ey * Ez[:, iz][:, None]).T @ Ex).real
        return amp * out

    kx = np.exp(field(facec, nodes, nodes))
    ky = np.exp(field(nodes, facec, nodes))
    kz = np.exp(field(nodes, nodes, facec))
    return kx, ky, kz


def manufactured_solution(dim: int, N: int) -> np.ndarray:
    """u_h = prod_d sin(pi x_d) at the interior nodes, x fastest."""
    h = 1.0 / (N + 1)
    s = np.sin(math.pi * (np.arange(N) + 1.0) * h)
    u = s
    for _ in range(dim - 1):
        u = np.multiply.outer(s, u)
    return np.ascontiguousarray(u.reshape(-1))


def rhs_from_solution(A: Csr, x: np.ndarray) -> np.ndarray:
    """b = A x in FP64 (scipy sparse product), so that x solves Ax = b up to
    the rounding of b."""
    return np.ascontiguousarray(A.to_scipy() @ np.asarray(x, dtype=np.float64))


def random_vector(n: int, seed: int, dist: str = "normal") -> np.ndarray:
    rng = np.random.default_rng(seed)
    if dist == "normal":
        return rng.standard_normal(n)
    if dist == "uniform":
        return rng.uniform(-1.0, 1.0, n)
    raise ValueError(dist)


def make_problem(dim: int, N: int, beta: float, rhs: str = "manufactured",
                 grf_seed: int | None = None, name: str | None = None) -> Problem:
    """One instance. rhs: 'ones' (b = A 1, exact solution 1, the paper's
    choice) or 'manufactured' (b = A u_h). grf_seed: None for k = 1, else the
    seed of the face-coefficient field (dim 3 only)."""
    faces = grf_faces(N, grf_seed) if grf_seed is not None else None
    A = convdiff_csr(dim, N, beta, faces)
    if rhs == "ones":
        xe = np.ones(A.n)
    elif rhs == "manufactured":
        xe = manufactured_solution(dim, N)
    else:
        raise ValueError(rhs)
    b = rhs_from_solution(A, xe)
    return Problem(name=name or f"{dim}d_N{N}_beta{beta:g}", dim=dim, N=N, beta=float(beta),
                   A=A, b=b, x_exact=xe, faces=faces)


def sylvester_matrices(n, r):
    """The tridiagonal test matrix of §4.3's Sylvester experiment, A = B =
    M + 2 r N + 100/(n+1)^2 I with M = tridiag(-1, 2, -1) and N =
    tridiag(0.5, 0, -0.5), as (lo, dg, up) with lo[i] = T[i][i-1], up[i] =
    T[i][i+1] (lo[0] and up[-1] are 0)."""
    lo = np.full(n, -1.0 + 2.0 * r * 0.5)
    up = np.full(n, -1.0 + 2.0 * r * (-0.5))
    dg = np.full(n, 2.0 + 100.0 / (n + 1) ** 2)
    lo[0] = 0.0
    up[-1] = 0.0
    return lo, dg, up


def tri_dense(lo, dg, up):
    """The dense n x n matrix of a (lo, dg, up) tridiagonal triple."""
    n = len(dg)
    T = np.diag(dg).astype(np.float64)
    T[np.arange(1, n), np.arange(n - 1)] = lo[1:]
    T[np.arange(n - 1), np.arange(1, n)] = up[:-1]
    return T


def sylvester_problem(m, n, r, seed=0):
    """(a, b, X*, C) for A X + X B = C with the §4.3 matrices of sides m and
    n, X* standard normal (seeded), C = A X* + X* B in FP64."""
    a = sylvester_matrices(m, r)
    b = sylvester_matrices(n, r)
    Xs = np.random.default_rng(seed).standard_normal((m, n))
    A, B = tri_dense(*a), tri_dense(*b)
    return a, b, Xs, A @ Xs + Xs @ B


# The workloads: sizes, coefficients and right-hand sides of the paper's
# convection-diffusion experiment, at the grid sizes this library is measured on.
WORKLOADS = {
    # 2D 32x32, beta = 10, b = A*1; plain FP64 GADI anchor
    "convdiff2d_32_b10": dict(dim=2, N=32, beta=10.0, rhs="ones"),
    # 3D 64^3, beta = 100, manufactured sin solution
    "convdiff3d_64_b100": dict(dim=3, N=64, beta=100.0, rhs="manufactured"),
    # 3D 128^3, beta = 50, GRF face coefficients (seed 3), manufactured solution
    "convdiff3d_128_b50_grf": dict(dim=3, N=128, beta=50.0, rhs="manufactured", grf_seed=3),
    # 3D 160^3, beta = 100: a smaller system whose working set (about 0.3 GB)
    # still exceeds the 129 MB L2 (counter captures of the solve kernel)
    "convdiff3d_160_b100": dict(dim=3, N=160, beta=100.0, rhs="manufactured"),
    # 3D 192^3, beta = 100, manufactured solution: the working set (about 3 GB
    # with the solver's vectors) is many times the 129 MB L2, so the inner
    # sweeps stream from HBM
    "convdiff3d_192_b100": dict(dim=3, N=192, beta=100.0, rhs="manufactured"),
}


def workload(name: str) -> Problem:
    return make_problem(name=name, **WORKLOADS[name])
