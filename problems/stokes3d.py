"""3D Stokes, Taylor-Hood Q2-Q1 on jittered hexahedra with Dirichlet-trimmed
Vanka cell patches (input generator; none of the method's arithmetic).

* Mesh: N^3 cells of [0,1]^3; interior vertices moved by uniform(-j h, j h)^3
  (seeded), boundary vertices fixed; trilinear (Q1) geometry map, Q2 velocity
  and Q1 pressure defined on the reference cube.
* Velocity DOFs on the boundary are eliminated (not kept as identity rows), so
  cell patches have 3 x (free Q2 nodes of the cell) + 8 DOFs: 89 inside, 62 on
  faces, 44 on edges, 32 at corners.  Pressure DOF 0 (vertex (0,0,0)) is
  pinned with a unit row.
* Global numbering: u_x of the free Q2 nodes (lexicographic, x fastest), then
  u_y, u_z, then the (N+1)^3 pressure vertices.  Patch local order: free nodes
  of the cell in tensor order for u_x, u_y, u_z, then the 8 vertices.
* Element blocks (velocity stiffness, divergence) are formed per cell with
  batched products; the CSR assembly runs in native code (_assemble.c), row
  by row, each entry the sum of its cell contributions in increasing cell
  order, so the 48^3 case (about 4e8 stored entries) takes seconds.
"""
from __future__ import annotations

import numpy as np

from . import fem
from .configs import Problem


def _ref3d():
    phi, dphi, w = fem.tensor_basis(2, 3, 3)        # (27, 27q), (3, 27, 27q)
    psi, dpsi, _ = fem.tensor_basis(1, 3, 3)        # (8, 27q): pressure and geometry
    return phi, dphi, psi, dpsi, w


def _jittered_vertices(N: int, jitter: float, seed: int) -> np.ndarray:
    g = np.random.Generator(np.random.PCG64(seed))
    s = np.linspace(0.0, 1.0, N + 1)
    Z, Y, X = np.meshgrid(s, s, s, indexing="ij")
    V = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)
    h = 1.0 / N
    iz, iy, ix = np.meshgrid(np.arange(N + 1), np.arange(N + 1), np.arange(N + 1), indexing="ij")
    inner = ((ix > 0) & (ix < N) & (iy > 0) & (iy < N) & (iz > 0) & (iz < N)).reshape(-1)
    d = g.uniform(-jitter * h, jitter * h, size=V.shape)
    V[inner] += d[inner]
    return V


def _cell_mats(Xc, ref):
    """Velocity stiffness K (nc,27,27) and divergence blocks B (nc,3,8,27)
    for cells with vertex coordinates Xc (nc, 8, 3)."""
    phi, dphi, psi, dpsi, w = ref
    # J[c, q, i, j] = d x_i / d xi_j = sum_v X[c, v, i] dpsi[j, v, q]
    J = np.einsum("cvi,jvq->cqij", Xc, dpsi)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    # grad_x phi_a = J^{-T} grad_xi phi_a : G[c,q,a,i] = sum_j Jinv[c,q,j,i] dphi[j,a,q]
    G = np.einsum("cqji,jaq->cqai", Jinv, dphi)
    wd = w[None, :] * np.abs(det)
    nc, nq = wd.shape
    # K[c] = sum_{q,i} wd G G^T as one product per cell: H[c] = (sqrt(wd) G) laid
    # out (27 basis, nq * 3) so K[c] = H[c] H[c]^T
    H = np.ascontiguousarray(np.transpose(G * np.sqrt(wd)[:, :, None, None], (0, 2, 1, 3))).reshape(nc, 27, nq * 3)
    K = np.matmul(H, np.transpose(H, (0, 2, 1)))
    K = 0.5 * (K + np.transpose(K, (0, 2, 1)))
    # B[c, k, p, a] = -sum_q wd psi_p (G)_{a,k}: (8 x nq) @ (nq x 27*3) per cell
    Pw = psi[None, :, :] * wd[:, None, :]                       # (nc, 8, nq)
    B = -np.matmul(Pw, G.reshape(nc, nq, 27 * 3)).reshape(nc, 8, 27, 3)
    return K, np.ascontiguousarray(np.transpose(B, (0, 3, 1, 2)))


def stokes3d_q2q1(N: int = 48, jitter: float = 0.2, seed: int = 0, chunk_cells: int = 8192) -> Problem:
    from . import _native
    ref = _ref3d()
    V = _jittered_vertices(N, jitter, seed)
    m = 2 * N + 1                                   # Q2 nodes per direction
    nf = m - 2                                      # free nodes per direction
    nfree = nf ** 3
    nvert = (N + 1) ** 3
    n = 3 * nfree + nvert
    # free-node index of every Q2 node (-1 on the boundary)
    iz, iy, ix = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    ix = ix.reshape(-1); iy = iy.reshape(-1); iz = iz.reshape(-1)
    freeid = np.where((ix > 0) & (ix < m - 1) & (iy > 0) & (iy < m - 1) & (iz > 0) & (iz < m - 1),
                      (ix - 1) + nf * ((iy - 1) + nf * (iz - 1)), -1).astype(np.int64)
    cz, cy, cx = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    cx = cx.reshape(-1); cy = cy.reshape(-1); cz = cz.reshape(-1)
    nc = N ** 3
    # element DOF maps: 81 velocity (3 x 27, -1 if eliminated) + 8 pressure
    nodes = np.zeros((nc, 27), dtype=np.int64)
    for c in range(3):
        for b in range(3):
            for a in range(3):
                nodes[:, a + 3 * b + 9 * c] = (2 * cx + a) + m * ((2 * cy + b) + m * (2 * cz + c))
    fnodes = freeid[nodes]                          # (nc, 27)
    verts = np.zeros((nc, 8), dtype=np.int64)
    for c in range(2):
        for b in range(2):
            for a in range(2):
                verts[:, a + 2 * b + 4 * c] = (cx + a) + (N + 1) * ((cy + b) + (N + 1) * (cz + c))
    vel = [np.where(fnodes >= 0, k * nfree + fnodes, -1) for k in range(3)]
    edofs = np.ascontiguousarray(np.concatenate(vel + [3 * nfree + verts], axis=1))  # (nc, 89), -1 = eliminated
    pin = 3 * nfree                                                   # pressure vertex 0
    # patches: the cell's kept DOFs in element order
    keep = edofs >= 0
    sizes = keep.sum(axis=1)
    offsets = np.zeros(nc + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    flat = edofs[keep]
    # element blocks of every cell (in chunks), then CSR assembly in native
    # code: row by row, cell contributions summed in increasing cell order
    K = np.empty((nc, 27, 27))
    B = np.empty((nc, 3, 8, 27))
    for c0 in range(0, nc, chunk_cells):
        c1 = min(nc, c0 + chunk_cells)
        K[c0:c1], B[c0:c1] = _cell_mats(V[verts[c0:c1]], ref)
    lib = _native.lib()
    rowptr = np.zeros(n + 1, dtype=np.int64)
    if lib.stokes3d_pattern_count(n, nc, edofs.ctypes.data, pin, rowptr.ctypes.data) != 0:
        raise MemoryError("stokes3d assembly: out of host memory (pattern)")
    if rowptr[-1] >= 2 ** 31:
        raise ValueError("nnz exceeds int32")
    cols = np.empty(int(rowptr[-1]), dtype=np.int32)
    vals = np.empty(int(rowptr[-1]), dtype=np.float64)
    if lib.stokes3d_fill(n, nc, edofs.ctypes.data, pin, rowptr.ctypes.data, K.ctypes.data, B.ctypes.data,
                         cols.ctypes.data, vals.ctypes.data) != 0:
        raise MemoryError("stokes3d assembly: out of host memory (values)")
    del K, B
    rhs_mask = np.zeros(n, dtype=bool)
    rhs_mask[:3 * nfree] = True
    return Problem(f"stokes3d_q2q1_N{N}", n, rowptr.astype(np.int32), cols, vals,
                   offsets.astype(np.int32), flat.astype(np.int32), rhs_mask,
                   symmetric=True, krylov="fgmres", weighting="left",
                   meta={"N": N, "jitter": jitter, "seed": seed, "sizes": sorted(set(sizes.tolist()))})
