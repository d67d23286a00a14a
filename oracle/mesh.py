"""Structured quadrilateral / hexahedral meshes of the unit square / cube (oracle; test infrastructure).

The mesh is n^d cells with (n+1)^d vertices given as input (possibly perturbed); each cell
is mapped from the reference cell by the standard multilinear map T_K (Sec. 2.2, Def. VKQK).
Global numbering: cells and vertices lexicographic with x fastest.  Velocity DoFs are the
continuous Q_{r+1} nodes, N1 = (r+1) n + 1 per direction, component-major within one time
node; pressure DoFs are discontinuous, C(r+d,d) modes per cell, cell-major.
"""
import itertools

import numpy as np

from .reference import SpaceRef


class Mesh:
    def __init__(self, d, n, vertices):
        self.d, self.n = d, n
        self.vertices = np.asarray(vertices, float).reshape((n + 1) ** d, d)
        self.ncells = n ** d
        self.cell_multi = np.array(list(itertools.product(*([range(n)] * d))))[:, ::-1]

    def cell_vertices(self):
        """[ncells, 2^d, d] corner coordinates; corner c has bits (c>>l)&1 along axis l."""
        d, n = self.d, self.n
        out = np.zeros((self.ncells, 2 ** d, d))
        for c in range(2 ** d):
            off = np.array([(c >> l) & 1 for l in range(d)])
            vm = self.cell_multi + off
            vidx = np.zeros(self.ncells, int)
            stride = 1
            for l in range(d):
                vidx += vm[:, l] * stride
                stride *= n + 1
            out[:, c, :] = self.vertices[vidx]
        return out

    def map_points(self, ref_pts):
        """Physical points x = T_K(x_hat) [ncells, P, d] and Jacobians J[c,p,i,l] = dx_i/dx_hat_l."""
        d = self.d
        cv = self.cell_vertices()
        ref_pts = np.atleast_2d(ref_pts)
        P = len(ref_pts)
        N = np.ones((P, 2 ** d))
        dN = np.ones((P, 2 ** d, d))
        for c in range(2 ** d):
            for l in range(d):
                b = (c >> l) & 1
                val = ref_pts[:, l] if b else 1.0 - ref_pts[:, l]
                der = 1.0 if b else -1.0
                N[:, c] *= val
                for g in range(d):
                    dN[:, c, g] *= der if g == l else val
        x = np.einsum("pc,kci->kpi", N, cv)
        J = np.einsum("pcl,kci->kpil", dN, cv)
        return x, J

    @staticmethod
    def coarsen(mesh):
        """Coarse mesh of the hierarchy: every second vertex in each direction."""
        d, n = mesh.d, mesh.n
        assert n % 2 == 0
        V = mesh.vertices.reshape(*([n + 1] * d), d)
        sl = tuple([slice(None, None, 2)] * d)
        return Mesh(d, n // 2, V[sl].reshape(-1, d))


def uniform_vertices(d, n):
    """Vertices of the uniform n^d grid on [0,1]^d, x fastest."""
    g = np.linspace(0.0, 1.0, n + 1)
    pts = np.array(list(itertools.product(*([g] * d))))[:, ::-1]
    return pts


class Space:
    """Q_{r+1}^d x P_r^disc on a mesh: DoF maps and geometry at quadrature points."""

    def __init__(self, mesh, r, nq=None):
        self.mesh = mesh
        self.d, self.r = mesh.d, r
        self.ref = SpaceRef(mesh.d, r, nq)
        d, n = self.d, mesh.n
        self.N1 = (r + 1) * n + 1
        self.nnodes = self.N1 ** d
        self.Nv = d * self.nnodes
        self.npc = self.ref.np
        self.Np = mesh.ncells * self.npc
        # local node -> global node index [ncells, n_loc]
        loc = self.ref.local_node_multi()
        gm = mesh.cell_multi[:, None, :] * (r + 1) + loc[None, :, :]
        stride = self.N1 ** np.arange(d)
        self.cell_nodes = np.einsum("cil,l->ci", gm, stride)
        # velocity dof (component c, local node i) -> global index within one time node
        self.nloc = loc.shape[0]
        self.cell_vdofs = np.concatenate(
            [self.cell_nodes + c * self.nnodes for c in range(d)], axis=1)   # [ncells, d*nloc]
        self.cell_pdofs = np.arange(self.Np).reshape(mesh.ncells, self.npc)
        # geometry at volume quadrature points
        self.xq, J = mesh.map_points(self.ref.qpts)
        self.detJ = np.linalg.det(J)
        assert np.all(self.detJ > 0), "inverted cell"
        self.G = np.linalg.inv(J)                             # G[c,q,m,i] = dxhat_m/dx_i
        self.JxW = self.detJ * self.ref.qwts[None, :]
        # physical gradients of the velocity basis [ncells, Q, nloc, d]
        self.gphi = np.einsum("qjm,cqmi->cqji", self.ref.dphi, self.G)
        self.cell_volume = self.JxW.sum(axis=1)
        self._faces()

    def _faces(self):
        """Boundary faces: (cell, axis, side) with geometry at face quadrature points."""
        d, n = self.d, self.mesh.n
        faces = []
        for axis in range(d):
            for side in (0, 1):
                cells = np.nonzero(self.mesh.cell_multi[:, axis] == (0 if side == 0 else n - 1))[0]
                for c in cells:
                    faces.append((c, axis, side))
        self.faces = faces
        self.face_data = {}
        for axis in range(d):
            for side in (0, 1):
                pts, wts = self.ref.face_points(axis, side)
                phi, dphi = self.ref.velocity_basis(pts)
                psi = self.ref.pressure_basis(pts)
                x, J = self.mesh.map_points(pts)
                G = np.linalg.inv(J)
                detJ = np.linalg.det(J)
                nhat = np.zeros(d)
                nhat[axis] = 1.0 if side == 1 else -1.0
                # Nanson: n dS = det(J) J^{-T} nhat dS_hat
                cof = detJ[..., None] * np.einsum("cpmi,m->cpi", G, nhat)
                dS = np.linalg.norm(cof, axis=2)
                nrm = cof / dS[..., None]
                gphi = np.einsum("pjm,cpmi->cpji", dphi, G)
                self.face_data[(axis, side)] = dict(
                    phi=phi, psi=psi, x=x, normal=nrm, JxW=dS * wts[None, :], gphi=gphi)

    def face_h(self, cell, axis, side):
        """h_F = |K| / |F| (reading of the undefined h_{Gamma_D} of Eq. def-b-gam-3)."""
        fd = self.face_data[(axis, side)]
        return self.cell_volume[cell] / fd["JxW"][cell].sum()

    def node_coords(self):
        """Physical coordinates of all global velocity nodes [nnodes, d]."""
        d = self.d
        X = np.zeros((self.nnodes, d))
        ref_nodes = np.array(list(itertools.product(*([self.ref.nodes] * d))))[:, ::-1]
        x, _ = self.mesh.map_points(ref_nodes)
        for c in range(self.mesh.ncells):
            X[self.cell_nodes[c]] = x[c]
        return X

    def sizes(self, k):
        return self.Nv, self.Np, (k + 1) * (self.Nv + self.Np)
