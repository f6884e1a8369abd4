"""Seeded synthetic pencils and blocks (shared by tests, bench and smoke).

This module builds problem inputs only: the sparse Hermitian-definite pencils
(A, B) the paper's numerical section works on, random starting blocks and the
interval bookkeeping.  It contains none of the eigensolver's arithmetic
(no filter, no factorisation, no Krylov step), so both the CUDA path and the
CPU oracle may consume what it produces.

Grid convention: vertex id  v = x + nx*(y + ny*z)  (x fastest), 0-based.
The Laplacian is unscaled: 2*d on the diagonal, -1 on each nearest neighbour
(Dirichlet), so its 1D factor has eigenvalues 2 - 2 cos(i pi/(n+1)).
Random numbers come from numpy's PCG64 ``default_rng(seed)``.
"""
import math
import numpy as np
import scipy.sparse as sp


def _lap1d(n):
    return sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")


def _mass1d(n):
    """1D linear-FE mass stencil [1/6, 2/3, 1/6] (row sums 1 away from the boundary)."""
    return sp.diags([np.full(n - 1, 1.0 / 6.0), np.full(n, 2.0 / 3.0), np.full(n - 1, 1.0 / 6.0)],
                    [-1, 0, 1], format="csr")


def _eye(n):
    return sp.identity(n, format="csr")


def _kron3(Tz, Ty, Tx):
    return sp.kron(Tz, sp.kron(Ty, Tx, format="csr"), format="csr")


def laplacian(dims, phase=0.0):
    """Nearest-neighbour Laplacian on a 1D/2D/3D grid, optional Peierls phase.

    With ``phase`` = theta, the hopping on the x-link from x to x+1 at row y is
    -exp(i theta y) (and its conjugate on the reverse link), which keeps A Hermitian.
    """
    dims = tuple(int(d) for d in dims)
    nx = dims[0]
    ny = dims[1] if len(dims) > 1 else 1
    nz = dims[2] if len(dims) > 2 else 1
    n = nx * ny * nz
    Ix, Iy, Iz = _eye(nx), _eye(ny), _eye(nz)
    Ly = _kron3(Iz, _lap1d(ny), Ix) if ny > 1 else sp.csr_matrix((n, n))
    Lz = _kron3(_lap1d(nz), Iy, Ix) if nz > 1 else sp.csr_matrix((n, n))
    if phase == 0.0:
        Lx = _kron3(Iz, Iy, _lap1d(nx))
        A = (Lx + Ly + Lz).astype(np.float64)
    else:
        idx = np.arange(n)
        x = idx % nx
        y = (idx // nx) % ny
        m = x < nx - 1
        i = idx[m]
        hop = -np.exp(1j * phase * y[m])
        off = sp.csr_matrix((hop, (i, i + 1)), shape=(n, n))
        Lx = sp.diags(np.full(n, 2.0 + 0j)) + off + off.conj().T
        A = (Lx + Ly + Lz).astype(np.complex128)
    return A.tocsr()


def mass_x(dims, weight=0.1):
    """B = I + weight * (1D mass stencil along x)  (configuration of the 2D/3D real pencils)."""
    dims = tuple(int(d) for d in dims)
    nx = dims[0]
    ny = dims[1] if len(dims) > 1 else 1
    nz = dims[2] if len(dims) > 2 else 1
    n = nx * ny * nz
    return (_eye(n) + weight * _kron3(_eye(nz), _eye(ny), _mass1d(nx))).tocsr()


def mass_trilinear(dims):
    """27-point trilinear finite-element mass matrix M1 (x) M1 (x) M1, row sums 1 inside."""
    nx, ny, nz = (int(d) for d in dims)
    return _kron3(_mass1d(nz), _mass1d(ny), _mass1d(nx)).tocsr()


def gaussian_wells(dims, count, rng, depth=(-5.0, 0.0), width=(1.0, 4.0)):
    """Sum of ``count`` Gaussians d*exp(-|r-c|^2/(2w^2)), d~U[depth], w~U[width], c~U[0,n)^3."""
    nx, ny, nz = (int(d) for d in dims)
    d = rng.uniform(depth[0], depth[1], size=count)
    w = rng.uniform(width[0], width[1], size=count)
    c = rng.uniform(0.0, 1.0, size=(count, 3)) * np.array([nx, ny, nz], dtype=np.float64)
    n = nx * ny * nz
    idx = np.arange(n)
    x = (idx % nx).astype(np.float64)
    y = ((idx // nx) % ny).astype(np.float64)
    z = (idx // (nx * ny)).astype(np.float64)
    V = np.zeros(n)
    for t in range(count):
        r2 = (x - c[t, 0]) ** 2 + (y - c[t, 1]) ** 2 + (z - c[t, 2]) ** 2
        V += d[t] * np.exp(-r2 / (2.0 * w[t] ** 2))
    return V


class Pencil:
    """A sparse pencil (A, B) on a grid, with the recipe that made it."""

    def __init__(self, A, B, dims, name, recipe):
        self.A = A.tocsr()
        self.B = B.tocsr()
        self.A.sort_indices()
        self.B.sort_indices()
        self.dims = tuple(dims)
        self.name = name
        self.recipe = recipe

    @property
    def n(self):
        return self.A.shape[0]

    @property
    def is_complex(self):
        return np.iscomplexobj(self.A.data) or np.iscomplexobj(self.B.data)


def pencil_2d_real(n=40, seed=1, vmax=2.0):
    """2D 5-point Laplacian n x n + diag U[0,vmax]; B = I + 0.1 (mass stencil along x)."""
    rng = np.random.default_rng(seed)
    dims = (n, n)
    V = rng.uniform(0.0, vmax, size=n * n)
    A = laplacian(dims) + sp.diags(V)
    B = mass_x(dims)
    return Pencil(A, B, dims, f"lap2d_{n}x{n}_real", f"seed={seed}; V~U[0,{vmax}]; B=I+0.1*M1x")


def pencil_3d_real(n, seed, vmax=2.0, b_diag=None):
    """3D 7-point Laplacian n^3 + diag U[0,vmax]; B = I + 0.1 M1x, or diag U[b_diag] if given."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    V = rng.uniform(0.0, vmax, size=n ** 3)
    A = laplacian(dims) + sp.diags(V)
    if b_diag is None:
        B = mass_x(dims)
        bdesc = "I+0.1*M1x"
    else:
        B = sp.diags(rng.uniform(b_diag[0], b_diag[1], size=n ** 3)).tocsr()
        bdesc = f"diag U{list(b_diag)}"
    return Pencil(A, B, dims, f"lap3d_{n}^3_real", f"seed={seed}; V~U[0,{vmax}]; B={bdesc}")


def pencil_3d_peierls(n=64, seed=2, theta=0.05, wells=32):
    """Complex Hermitian 3D pencil: Peierls-phase 7-point Laplacian + Gaussian wells;
    B = normalised 27-point trilinear mass (SPD, eigenvalues in (1/27, 1))."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    V = gaussian_wells(dims, wells, rng)
    A = laplacian(dims, phase=theta) + sp.diags(V.astype(np.complex128))
    B = mass_trilinear(dims)
    return Pencil(A, B, dims, f"peierls3d_{n}^3",
                  f"seed={seed}; theta={theta}; {wells} wells d~U[-5,0] w~U[1,4]; B=M1^(x3)")


def hamiltonian_wells(n, seed, wells=3, radius=0.2):
    """The 3D Hamiltonian H = -1/2 Laplacian + V of Section 3.1 (Example 1) on the unit cube
    with a Dirichlet boundary: n interior points per axis at x_i = i h, i = 1..n,
    h = 1/(n+1), the 7-point finite-difference Laplacian (so -1/2 Laplacian has 3/h^2 on
    the diagonal and -1/(2h^2) on each neighbour), and V = sum of ``wells`` Gaussian wells
    -d exp(-|r - c|^2 / (2 radius^2)) with depth d uniform in (0, 1] and centre c uniform
    in [0, 1)^3.  B = I.  Returned as a real pencil on the (n, n, n) grid."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    h = 1.0 / (n + 1)
    d = 1.0 - rng.uniform(0.0, 1.0, size=wells)          # (0, 1]
    c = rng.uniform(0.0, 1.0, size=(wells, 3))
    idx = np.arange(n ** 3)
    x = (idx % n + 1) * h
    y = ((idx // n) % n + 1) * h
    z = (idx // (n * n) + 1) * h
    V = np.zeros(n ** 3)
    for t in range(wells):
        r2 = (x - c[t, 0]) ** 2 + (y - c[t, 1]) ** 2 + (z - c[t, 2]) ** 2
        V -= d[t] * np.exp(-r2 / (2.0 * radius ** 2))
    A = (laplacian(dims) * (0.5 / h ** 2) + sp.diags(V)).tocsr()
    B = _eye(n ** 3)
    return Pencil(A, B, dims, f"ham3d_{n}^3_wells",
                  f"seed={seed}; -1/2 Laplacian (h=1/{n + 1}) + {wells} wells d~U(0,1] radius {radius}; B=I")


def random_block(n, k, seed, complex_=True):
    """N x k starting block with standard normal entries (complex: (N(0,1)+iN(0,1))/sqrt 2),
    row-major (k fastest)."""
    rng = np.random.default_rng(1_000_003 + int(seed))
    if complex_:
        return ((rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))) / math.sqrt(2.0))
    return rng.standard_normal((n, k))


def csr_arrays(M, complex_=True):
    """(row_ptr int64, col_idx int32, values) of a scipy CSR matrix, indices sorted."""
    M = M.tocsr()
    M.sort_indices()
    vals = M.data.astype(np.complex128 if complex_ else np.float64)
    return M.indptr.astype(np.int64), M.indices.astype(np.int32), np.ascontiguousarray(vals)
