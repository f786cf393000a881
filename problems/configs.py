"""Seeded synthetic workloads: assembled CSR matrix + cell -> DOF patch map.

Five families, each parameterised by mesh size so that tests can use tiny
instances of exactly the same structure as the full-size workloads:

* ``poisson2d_q2``   -- 2D scalar diffusion, Q2 Lagrange, uniform N x N quads of
  [0,1]^2, rho = 1, homogeneous Dirichlet (identity rows); 9-DOF cell patches.
  Full size: N = 16 (1,089 DOFs, 256 patches).
* ``stokes2d_q2q1``  -- 2D Stokes, Taylor-Hood Q2-Q1, N x N quads graded
  geometrically in y (ratio 1.05, finest at y = 0), all-Dirichlet velocity,
  pressure DOF 0 pinned; 22-DOF cell (Vanka) patches.  Full size: N = 128.
* ``nedelec3d``      -- 3D curl(nu curl u) + alpha u, lowest-order Nedelec hexes
  on N^3 cells of [0,1]^3, nu ~ lognormal(0, 0.5) per cell, alpha = 1e-3,
  tangential trace 0 on the boundary; 12-DOF patches.  Full size: N = 64.
* ``diffusion3d_q2`` -- 3D scalar diffusion, Q2 on N^3 cells, lognormal
  coefficient (sigma = 1, correlation length 8 cells, Gaussian-filtered
  noise); 27-DOF patches.  Full size: N = 32.
* ``stokes3d_q2q1``  -- 3D Stokes Q2-Q1 on jittered N^3 hexes (interior vertex
  displacement uniform in [-0.2h, 0.2h]^3, trilinear geometry), Dirichlet
  velocity DOFs eliminated ("trimmed"), pressure DOF 0 pinned; patches of
  89/62/44/32 DOFs.  Full size: N = 48.

Nothing here is part of the patch-relaxation method; it only builds inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import fem


@dataclass
class Problem:
    name: str
    n: int
    rowptr: np.ndarray          # int32 [n+1]
    colidx: np.ndarray          # int32 [nnz], sorted + unique per row
    vals: np.ndarray            # float64 [nnz]
    patch_offsets: np.ndarray   # int32 [n_patches+1]
    patch_dofs: np.ndarray      # int32 [sum p_s], flat, cell (lexicographic) order
    rhs_mask: np.ndarray        # bool [n]: rows that receive a random rhs entry
    symmetric: bool
    krylov: str                 # "cg" | "fgmres"
    weighting: str              # "sym" | "left"
    meta: dict = field(default_factory=dict)
    cell_coef: np.ndarray | None = None   # per-cell coefficient (feature input)

    @property
    def nnz(self) -> int:
        return int(self.colidx.size)

    @property
    def n_patches(self) -> int:
        return int(self.patch_offsets.size - 1)

    @property
    def patch_sizes(self) -> np.ndarray:
        return np.diff(self.patch_offsets)

    @property
    def uniform_size(self) -> int:
        s = self.patch_sizes
        return int(s[0]) if s.size and np.all(s == s[0]) else 0

    def dofs2d(self) -> np.ndarray:
        p = self.uniform_size
        assert p > 0, "patches of uneven size"
        return self.patch_dofs.reshape(self.n_patches, p)

    def rhs(self, seed: int) -> np.ndarray:
        """uniform(-1, 1) on the rows of rhs_mask, 0 elsewhere (PCG64(seed))."""
        g = np.random.Generator(np.random.PCG64(seed))
        b = np.zeros(self.n)
        m = self.rhs_mask
        b[m] = g.uniform(-1.0, 1.0, size=int(m.sum()))
        return b

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals, self.colidx, self.rowptr), shape=(self.n, self.n))


def _uniform_patches(dofs: np.ndarray):
    nc, p = dofs.shape
    return (np.arange(nc + 1, dtype=np.int64) * p).astype(np.int32), dofs.astype(np.int32).reshape(-1)


# --------------------------------------------------------------------------
# 2D helpers
# --------------------------------------------------------------------------

def _q2_cell_nodes_2d(nx: int, ny: int) -> np.ndarray:
    """(nx*ny, 9) Q2 node ids per cell; cells x-fastest, local nodes x-fastest."""
    cx, cy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    cx = cx.reshape(-1)
    cy = cy.reshape(-1)
    stride = 2 * nx + 1
    out = np.zeros((nx * ny, 9), dtype=np.int64)
    for b in range(3):
        for a in range(3):
            out[:, a + 3 * b] = (2 * cx + a) + stride * (2 * cy + b)
    return out


def _q1_cell_vertices_2d(nx: int, ny: int) -> np.ndarray:
    cx, cy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    cx = cx.reshape(-1)
    cy = cy.reshape(-1)
    stride = nx + 1
    out = np.zeros((nx * ny, 4), dtype=np.int64)
    for b in range(2):
        for a in range(2):
            out[:, a + 2 * b] = (cx + a) + stride * (cy + b)
    return out


def _boundary_nodes_2d(nnx: int, nny: int) -> np.ndarray:
    ix, iy = np.meshgrid(np.arange(nnx), np.arange(nny), indexing="xy")
    return ((ix == 0) | (ix == nnx - 1) | (iy == 0) | (iy == nny - 1)).reshape(-1)


def graded_sizes(n: int, ratio: float) -> np.ndarray:
    """Cell sizes h_j = h0 * ratio^j, j = 0..n-1, summing to 1."""
    if ratio == 1.0:
        return np.full(n, 1.0 / n)
    h0 = (ratio - 1.0) / (ratio ** n - 1.0)
    return h0 * ratio ** np.arange(n)


def poisson2d_q2(N: int = 16, rho: float = 1.0, keep_pattern: bool = False) -> Problem:
    """2D Q2 diffusion on a uniform N x N mesh with Dirichlet identity rows
    (keep_pattern: their couplings stay stored as zeros)."""
    Kdir, _ = fem.reference_matrices(2, 2, 3)
    nc = N * N
    h = np.full((nc, 2), 1.0 / N)
    Ke = fem.rect_diffusion_element(Kdir, h, np.full(nc, rho))
    edofs = _q2_cell_nodes_2d(N, N)
    n = (2 * N + 1) ** 2
    bnd = _boundary_nodes_2d(2 * N + 1, 2 * N + 1)
    rowptr, colidx, vals = fem.assemble_csr(n, edofs, Ke, bnd, keep_pattern=keep_pattern)
    off, flat = _uniform_patches(edofs)
    return Problem(f"poisson2d_q2_N{N}", n, rowptr, colidx, vals, off, flat, ~bnd,
                   symmetric=True, krylov="cg", weighting="sym",
                   meta={"N": N, "p_s": 9, "dirichlet": bnd})


def _qp_cell_nodes_2d(N: int, p: int) -> np.ndarray:
    """(N*N, (p+1)^2) node ids of Q_p cells on the (Np+1)^2 node grid; cells
    x-fastest, local nodes x-fastest."""
    cx, cy = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    cx = cx.reshape(-1)
    cy = cy.reshape(-1)
    stride = N * p + 1
    n1 = p + 1
    out = np.zeros((N * N, n1 * n1), dtype=np.int64)
    for b in range(n1):
        for a in range(n1):
            out[:, a + n1 * b] = (p * cx + a) + stride * (p * cy + b)
    return out


def smooth2d_qp(N: int = 60, p: int = 2) -> Problem:
    """Experiment 1 of the paper (section 4): -div(rho grad u) = f on the unit
    square, rho = sin^2(pi x) sin^2(pi y) + 0.1 (evaluated at the quadrature
    points), f such that u = sin(pi x) sin(pi y), homogeneous Dirichlet
    (identity rows), Q_p elements (equispaced nodes) on a uniform N x N mesh;
    one patch per cell ((p+1)^2 DOFs).

    meta["P0"]: the linear (bilinear) interpolation from the (N+1)^2 mesh
    vertices to the (Np+1)^2 nodes, which the paper's two-level preconditioner
    uses with R0 = P0^T, as (rowptr, colidx, vals, n0) of an n x n0 CSR;
    meta["b"]: the load vector of f (0 on Dirichlet rows); meta["u_nodes"]:
    the exact solution at the nodes."""
    nq = p + 2
    xq, wq = fem.gauss_legendre_01(nq)
    phi, dphi, w = fem.tensor_basis(p, 2, nq)
    h = 1.0 / N
    nb = (p + 1) ** 2
    nqt = nq * nq
    qx = np.array([xq[q % nq] for q in range(nqt)])
    qy = np.array([xq[q // nq] for q in range(nqt)])
    edofs = _qp_cell_nodes_2d(N, p)
    cx = np.tile(np.arange(N), N)
    cy = np.repeat(np.arange(N), N)
    X = (cx[:, None] + qx[None, :]) * h                 # (nc, nqt) physical points
    Y = (cy[:, None] + qy[None, :]) * h
    sx, sy = np.sin(np.pi * X), np.sin(np.pi * Y)
    kx, ky = np.cos(np.pi * X), np.cos(np.pi * Y)
    rho = sx ** 2 * sy ** 2 + 0.1
    # f = -(grad rho . grad u + rho lap u), u = sin sin, lap u = -2 pi^2 u
    drx = 2.0 * np.pi * sx * kx * sy ** 2
    dry = 2.0 * np.pi * sx ** 2 * sy * ky
    ux = np.pi * kx * sy
    uy = np.pi * sx * ky
    f = -(drx * ux + dry * uy) + rho * 2.0 * np.pi ** 2 * sx * sy
    # element matrices: sum_q w_q rho_q (dphi_x dphi_x + dphi_y dphi_y) (h^2 / h^2)
    wr = rho * w[None, :]
    Ke = np.einsum("cq,aq,bq->cab", wr, dphi[0], dphi[0]) + np.einsum("cq,aq,bq->cab", wr, dphi[1], dphi[1])
    Ke = 0.5 * (Ke + np.transpose(Ke, (0, 2, 1)))
    fe = np.einsum("cq,aq->ca", f * w[None, :], phi) * (h * h)
    nn = N * p + 1
    n = nn * nn
    bnd = _boundary_nodes_2d(nn, nn)
    rowptr, colidx, vals = fem.assemble_csr(n, edofs, Ke, bnd)
    b = np.zeros(n)
    np.add.at(b, edofs.reshape(-1), fe.reshape(-1))
    b[bnd] = 0.0
    off, flat = _uniform_patches(edofs)
    # P0: node (i, j) of the fine grid from the vertices of the coarse cell
    # holding it, bilinear weights; exact zeros dropped
    ii, jj = np.meshgrid(np.arange(nn), np.arange(nn), indexing="xy")
    ii, jj = ii.reshape(-1), jj.reshape(-1)
    ci = np.minimum(ii // p, N - 1)
    cj = np.minimum(jj // p, N - 1)
    s_ = (ii - ci * p) / p
    t_ = (jj - cj * p) / p
    nv = N + 1
    cols = [ci + nv * cj, ci + 1 + nv * cj, ci + nv * (cj + 1), ci + 1 + nv * (cj + 1)]
    wts = [(1 - s_) * (1 - t_), s_ * (1 - t_), (1 - s_) * t_, s_ * t_]
    rows_l, cols_l, vals_l = [], [], []
    for cc, ww in zip(cols, wts):
        m = ww != 0.0
        rows_l.append(np.flatnonzero(m))
        cols_l.append(cc[m])
        vals_l.append(ww[m])
    r_ = np.concatenate(rows_l)
    c_ = np.concatenate(cols_l)
    v_ = np.concatenate(vals_l)
    order = np.lexsort((c_, r_))
    r_, c_, v_ = r_[order], c_[order], v_[order]
    prow = np.zeros(n + 1, dtype=np.int64)
    np.add.at(prow, r_ + 1, 1)
    prow = np.cumsum(prow)
    u_nodes = np.sin(np.pi * ii / (nn - 1)) * np.sin(np.pi * jj / (nn - 1))
    return Problem(f"smooth2d_q{p}_N{N}", n, rowptr, colidx, vals, off, flat, ~bnd,
                   symmetric=True, krylov="fgmres", weighting="left",
                   meta={"N": N, "p": p, "p_s": nb, "dirichlet": bnd, "b": b, "u_nodes": u_nodes,
                         "P0": (prow.astype(np.int32), c_.astype(np.int32), v_.astype(np.float64), nv * nv)})


def stokes2d_q2q1(N: int = 128, ratio: float = 1.05, keep_pattern: bool = False) -> Problem:
    """2D Taylor-Hood Stokes [K B^T; B 0] on an N x N mesh graded in y
    (keep_pattern: Dirichlet couplings stay stored as zeros)."""
    Kdir, _ = fem.reference_matrices(2, 2, 3)
    Bref = fem.reference_divergence(2, 1, 2, 3)          # (2, 4, 9)
    hx = np.full(N, 1.0 / N)
    hy = graded_sizes(N, ratio)
    HX, HY = np.meshgrid(hx, hy, indexing="xy")
    h = np.stack([HX.reshape(-1), HY.reshape(-1)], axis=1)
    nc = N * N
    K = fem.rect_diffusion_element(Kdir, h, np.ones(nc))  # (nc, 9, 9)
    vol = h[:, 0] * h[:, 1]
    Bx = -(vol / h[:, 0])[:, None, None] * Bref[0][None]  # (nc, 4, 9)
    By = -(vol / h[:, 1])[:, None, None] * Bref[1][None]
    E = np.zeros((nc, 22, 22))
    E[:, 0:9, 0:9] = K
    E[:, 9:18, 9:18] = K
    E[:, 18:22, 0:9] = Bx
    E[:, 18:22, 9:18] = By
    E[:, 0:9, 18:22] = np.transpose(Bx, (0, 2, 1))
    E[:, 9:18, 18:22] = np.transpose(By, (0, 2, 1))
    nodes = _q2_cell_nodes_2d(N, N)
    verts = _q1_cell_vertices_2d(N, N)
    nv = (2 * N + 1) ** 2
    npv = (N + 1) ** 2
    edofs = np.concatenate([nodes, nv + nodes, 2 * nv + verts], axis=1)
    n = 2 * nv + npv
    bnd = _boundary_nodes_2d(2 * N + 1, 2 * N + 1)
    dirichlet = np.zeros(n, dtype=bool)
    dirichlet[:nv] = bnd
    dirichlet[nv:2 * nv] = bnd
    dirichlet[2 * nv] = True            # pressure pin at vertex (0, 0)
    rowptr, colidx, vals = fem.assemble_csr(n, edofs, E, dirichlet, keep_pattern=keep_pattern)
    rhs_mask = np.zeros(n, dtype=bool)
    rhs_mask[:2 * nv] = ~dirichlet[:2 * nv]
    off, flat = _uniform_patches(edofs)
    return Problem(f"stokes2d_q2q1_N{N}", n, rowptr, colidx, vals, off, flat, rhs_mask,
                   symmetric=True, krylov="fgmres", weighting="left",
                   meta={"N": N, "ratio": ratio, "p_s": 22, "dirichlet": dirichlet,
                         "hy": hy})


# --------------------------------------------------------------------------
# 3D helpers
# --------------------------------------------------------------------------

def _cells3d(N: int):
    cz, cy, cx = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    return cx.reshape(-1), cy.reshape(-1), cz.reshape(-1)


def _q2_cell_nodes_3d(N: int) -> np.ndarray:
    cx, cy, cz = _cells3d(N)
    s = 2 * N + 1
    out = np.zeros((N ** 3, 27), dtype=np.int64)
    for c in range(3):
        for b in range(3):
            for a in range(3):
                out[:, a + 3 * b + 9 * c] = (2 * cx + a) + s * ((2 * cy + b) + s * (2 * cz + c))
    return out


def _q1_cell_vertices_3d(N: int) -> np.ndarray:
    cx, cy, cz = _cells3d(N)
    s = N + 1
    out = np.zeros((N ** 3, 8), dtype=np.int64)
    for c in range(2):
        for b in range(2):
            for a in range(2):
                out[:, a + 2 * b + 4 * c] = (cx + a) + s * ((cy + b) + s * (cz + c))
    return out


def _boundary_nodes_3d(m: int) -> np.ndarray:
    iz, iy, ix = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    b = (ix == 0) | (ix == m - 1) | (iy == 0) | (iy == m - 1) | (iz == 0) | (iz == m - 1)
    return b.reshape(-1)


def gaussian_random_field(N: int, corr_len: float, seed: int) -> np.ndarray:
    """Unit-variance Gaussian field on N^3 cells: white noise N(0,1) convolved
    (periodically) with a Gaussian kernel of std corr_len/sqrt(2) cells,
    truncated at 4 std, normalised by the kernel's l2 norm.  Cells x-fastest."""
    g = np.random.Generator(np.random.PCG64(seed))
    noise = g.standard_normal((N, N, N))          # indexed [z, y, x]
    s = corr_len / np.sqrt(2.0)
    r = int(np.ceil(4.0 * s))
    offs = np.arange(-r, r + 1)
    k1 = np.exp(-0.5 * (offs / s) ** 2)
    kern = np.zeros((N, N, N))
    for dz, wz in zip(offs, k1):
        for dy, wy in zip(offs, k1):
            for dx, wx in zip(offs, k1):
                kern[dz % N, dy % N, dx % N] += wz * wy * wx
    field_ = np.real(np.fft.ifftn(np.fft.fftn(noise) * np.fft.fftn(kern)))
    field_ /= np.sqrt(np.sum(kern ** 2))
    return field_.reshape(-1)


def diffusion3d_q2(N: int = 32, sigma: float = 1.0, corr_len: float = 8.0, seed: int = 0,
                   uniform: bool = False, keep_pattern: bool = False) -> Problem:
    """3D Q2 diffusion with a lognormal cell coefficient (or rho = 1 when
    uniform=True), Dirichlet identity rows; 27-DOF patches."""
    Kdir, _ = fem.reference_matrices(2, 3, 3)
    nc = N ** 3
    if uniform:
        rho = np.ones(nc)
    else:
        rho = np.exp(sigma * gaussian_random_field(N, corr_len, seed))
    h = np.full((nc, 3), 1.0 / N)
    Ke = fem.rect_diffusion_element(Kdir, h, rho)
    edofs = _q2_cell_nodes_3d(N)
    m = 2 * N + 1
    n = m ** 3
    bnd = _boundary_nodes_3d(m)
    rowptr, colidx, vals = fem.assemble_csr(n, edofs, Ke, bnd, keep_pattern=keep_pattern)
    off, flat = _uniform_patches(edofs)
    return Problem(f"diffusion3d_q2_N{N}", n, rowptr, colidx, vals, off, flat, ~bnd,
                   symmetric=True, krylov="cg", weighting="sym",
                   meta={"N": N, "p_s": 27, "sigma": sigma, "corr_len": corr_len,
                         "seed": seed, "uniform": uniform, "dirichlet": bnd},
                   cell_coef=rho)


# --------------------------------------------------------------------------
# Lowest-order Nedelec (edge) hexahedra
# --------------------------------------------------------------------------

def _nedelec_reference(nq: int = 2):
    """Values N[e, comp, q] and curls C[e, comp, q] of the 12 lowest-order
    Nedelec basis functions on the unit cube (before the 1/h scalings), local
    order: x-edges (b + 2c), y-edges 4 + (a + 2c), z-edges 8 + (a + 2b)."""
    xq, wq = fem.gauss_legendre_01(nq)
    Z, Y, X = np.meshgrid(xq, xq, xq, indexing="ij")
    X = X.reshape(-1); Y = Y.reshape(-1); Z = Z.reshape(-1)
    WZ, WY, WX = np.meshgrid(wq, wq, wq, indexing="ij")
    w = (WX * WY * WZ).reshape(-1)
    lin = [lambda t: 1.0 - t, lambda t: t]
    dlin = [-1.0, 1.0]
    nqt = X.size
    Nv = np.zeros((12, 3, nqt))
    # derivative factors dN[e][k] with respect to reference coordinate k
    dN = np.zeros((12, 3, 3, nqt))  # [e, comp, d/dk, q]
    for c in range(2):
        for b in range(2):
            e = b + 2 * c
            Nv[e, 0] = lin[b](Y) * lin[c](Z)
            dN[e, 0, 1] = dlin[b] * lin[c](Z)
            dN[e, 0, 2] = lin[b](Y) * dlin[c]
    for c in range(2):
        for a in range(2):
            e = 4 + a + 2 * c
            Nv[e, 1] = lin[a](X) * lin[c](Z)
            dN[e, 1, 0] = dlin[a] * lin[c](Z)
            dN[e, 1, 2] = lin[a](X) * dlin[c]
    for b in range(2):
        for a in range(2):
            e = 8 + a + 2 * b
            Nv[e, 2] = lin[a](X) * lin[b](Y)
            dN[e, 2, 0] = dlin[a] * lin[b](Y)
            dN[e, 2, 1] = lin[a](X) * dlin[b]
    return Nv, dN, w


def nedelec_element(h: np.ndarray, nu: np.ndarray, alpha: float) -> np.ndarray:
    """Element matrices nu_c int curl N_a . curl N_b + alpha int N_a . N_b for
    rectilinear hexes with sizes h (nc, 3) (covariant map: component k scaled
    by 1/h_k, derivative in k scaled by 1/h_k)."""
    Nv, dN, w = _nedelec_reference()
    nc = h.shape[0]
    out = np.zeros((nc, 12, 12))
    # physical field: F_comp = Nref_comp / h_comp ; d/dx_k = (1/h_k) d/dxhat_k
    # curl = (dF_z/dy - dF_y/dz, dF_x/dz - dF_z/dx, dF_y/dx - dF_x/dy)
    # vectorised over cells by grouping identical h (rectilinear uniform mesh)
    uh, inv = np.unique(h, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    for gi, hh in enumerate(uh):
        vol = hh[0] * hh[1] * hh[2]
        F = Nv / hh[None, :, None]
        dF = dN / hh[None, :, None, None] / hh[None, None, :, None]
        curl = np.stack([dF[:, 2, 1] - dF[:, 1, 2],
                         dF[:, 0, 2] - dF[:, 2, 0],
                         dF[:, 1, 0] - dF[:, 0, 1]], axis=1)
        Kc = np.einsum("q,ekq,fkq->ef", w, curl, curl) * vol
        Mm = np.einsum("q,ekq,fkq->ef", w, F, F) * vol
        Kc = 0.5 * (Kc + Kc.T)
        Mm = 0.5 * (Mm + Mm.T)
        sel = inv == gi
        out[sel] = nu[sel, None, None] * Kc[None] + alpha * Mm[None]
    return out


def nedelec3d(N: int = 64, nu_sigma: float = 0.5, alpha: float = 1e-3, seed: int = 0) -> Problem:
    """3D curl-curl + alpha mass on N^3 lowest-order Nedelec hexes."""
    nc = N ** 3
    g = np.random.Generator(np.random.PCG64(seed))
    nu = np.exp(nu_sigma * g.standard_normal(nc))
    h = np.full((nc, 3), 1.0 / N)
    Ke = nedelec_element(h, nu, alpha)
    cx, cy, cz = _cells3d(N)
    M = N + 1
    nxe = N * M * M
    edofs = np.zeros((nc, 12), dtype=np.int64)
    for c in range(2):
        for b in range(2):
            edofs[:, b + 2 * c] = cx + N * ((cy + b) + M * (cz + c))
    for c in range(2):
        for a in range(2):
            edofs[:, 4 + a + 2 * c] = nxe + (cx + a) + M * (cy + N * (cz + c))
    for b in range(2):
        for a in range(2):
            edofs[:, 8 + a + 2 * b] = 2 * nxe + (cx + a) + M * ((cy + b) + M * cz)
    n = 3 * nxe
    # boundary (tangential trace) edges
    bnd = np.zeros(n, dtype=bool)
    k, j, i = np.meshgrid(np.arange(M), np.arange(M), np.arange(N), indexing="ij")
    bnd[:nxe] = ((j == 0) | (j == N) | (k == 0) | (k == N)).reshape(-1)
    k, j, i = np.meshgrid(np.arange(M), np.arange(N), np.arange(M), indexing="ij")
    bnd[nxe:2 * nxe] = ((i == 0) | (i == N) | (k == 0) | (k == N)).reshape(-1)
    k, j, i = np.meshgrid(np.arange(N), np.arange(M), np.arange(M), indexing="ij")
    bnd[2 * nxe:] = ((i == 0) | (i == N) | (j == 0) | (j == N)).reshape(-1)
    rowptr, colidx, vals = fem.assemble_csr(n, edofs, Ke, bnd)
    off, flat = _uniform_patches(edofs)
    return Problem(f"nedelec3d_N{N}", n, rowptr, colidx, vals, off, flat, ~bnd,
                   symmetric=True, krylov="cg", weighting="sym",
                   meta={"N": N, "p_s": 12, "alpha": alpha, "nu_sigma": nu_sigma,
                         "seed": seed, "dirichlet": bnd},
                   cell_coef=nu)


BUILDERS = {
    "poisson2d_q2": poisson2d_q2,
    "stokes2d_q2q1": stokes2d_q2q1,
    "nedelec3d": nedelec3d,
    "diffusion3d_q2": diffusion3d_q2,
    "smooth2d_qp": smooth2d_qp,
}
