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
* Assembly runs in slabs of cell layers (rows of one slab of node layers are
  summed from the cells that touch them, in increasing cell order) so the
  48^3 case (about 4e8 nonzeros) fits in host memory.
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
    K = np.einsum("cq,cqai,cqbi->cab", wd, G, G)
    K = 0.5 * (K + np.transpose(K, (0, 2, 1)))
    B = -np.einsum("cq,pq,cqak->ckpa", wd, psi, G)
    return K, B


def stokes3d_q2q1(N: int = 48, jitter: float = 0.2, seed: int = 0, chunk_layers: int = 4) -> Problem:
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
    edofs = np.concatenate(vel + [3 * nfree + verts], axis=1)       # (nc, 89), -1 = eliminated
    pin = 3 * nfree                                                   # pressure vertex 0
    # patches: the cell's kept DOFs in element order
    keep = edofs >= 0
    sizes = keep.sum(axis=1)
    offsets = np.zeros(nc + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    flat = edofs[keep]
    # --- chunked assembly by slabs of cell layers
    rows_out, cols_out, vals_out = [], [], []
    layer_rows = []
    for z0 in range(0, N, chunk_layers):
        z1 = min(N, z0 + chunk_layers)
        # rows owned by this slab: velocity nodes with node-z in [2 z0, 2 z1) (last slab: up to m)
        # pressure vertices with z in [z0, z1) (last: up to N+1)
        nz_lo, nz_hi = 2 * z0, (2 * z1 if z1 < N else m)
        vz_lo, vz_hi = z0, (z1 if z1 < N else N + 1)
        cells = np.flatnonzero((cz >= max(z0 - 1, 0)) & (cz <= min(z1, N - 1)))
        Xc = V[verts[cells]]
        K, B = _cell_mats(Xc, ref)
        ncs = cells.size
        E = np.zeros((ncs, 89, 89))
        for k in range(3):
            E[:, 27 * k:27 * k + 27, 27 * k:27 * k + 27] = K
            E[:, 81:89, 27 * k:27 * k + 27] = B[:, k]
            E[:, 27 * k:27 * k + 27, 81:89] = np.transpose(B[:, k], (0, 2, 1))
        ed = edofs[cells]
        r = np.repeat(ed, 89, axis=1).reshape(-1)
        c = np.tile(ed, (1, 89)).reshape(-1)
        v = E.reshape(-1)
        del E
        ok = (r >= 0) & (c >= 0) & (r != pin) & (c != pin)
        # row ownership
        rv = np.where(r < 3 * nfree, r % nfree, 0)
        rnz = 1 + rv // (nf * nf)                          # node z of a free node
        own_v = (r < 3 * nfree) & (rnz >= nz_lo) & (rnz < nz_hi)
        rp = r - 3 * nfree
        own_p = (r >= 3 * nfree) & ((rp // ((N + 1) ** 2)) >= vz_lo) & ((rp // ((N + 1) ** 2)) < vz_hi)
        sel = ok & (own_v | own_p)
        r, c, v = r[sel], c[sel], v[sel]
        key = r * n + c
        order = np.argsort(key, kind="stable")      # cell order kept inside a key
        key = key[order]
        v = v[order]
        newg = np.empty(key.size, dtype=bool)
        if key.size:
            newg[0] = True
            np.not_equal(key[1:], key[:-1], out=newg[1:])
        starts = np.flatnonzero(newg)
        grp = np.cumsum(newg) - 1
        rank = np.arange(key.size) - starts[grp]
        sums = np.zeros(starts.size)
        for rr in range(int(rank.max()) + 1 if key.size else 0):
            mm = rank == rr
            sums[grp[mm]] += v[mm]
        uk = key[starts]
        rows_out.append(uk // n)
        cols_out.append(uk % n)
        vals_out.append(sums)
        del key, v, r, c, order, newg, grp, rank
    rows = np.concatenate(rows_out + [np.array([pin])])
    cols = np.concatenate(cols_out + [np.array([pin])])
    vals = np.concatenate(vals_out + [np.array([1.0])])
    o = np.lexsort((cols, rows))
    rows, cols, vals = rows[o], cols[o], vals[o]
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2 ** 31:
        raise ValueError("nnz exceeds int32")
    rhs_mask = np.zeros(n, dtype=bool)
    rhs_mask[:3 * nfree] = True
    return Problem(f"stokes3d_q2q1_N{N}", n, rowptr.astype(np.int32), cols.astype(np.int32), vals,
                   offsets.astype(np.int32), flat.astype(np.int32), rhs_mask,
                   symmetric=True, krylov="fgmres", weighting="left",
                   meta={"N": N, "jitter": jitter, "seed": seed, "sizes": sorted(set(sizes.tolist()))})
