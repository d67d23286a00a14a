"""Slab residual R_n, Jacobian J_n and mass-weighted norm (oracle; test infrastructure).

Follows Problem LocAlgNS (Sec. 3.3, Eq. InAlgNS) with the matrices of Appendix A
(Eq. DefMAB, DefNitscheSpatial1, DefNitscheSpatial10, DefFn, DefLn), the convective form in
divergence form (Eq. ns-form-tp), its Gateaux derivative (Eq. Defcp), the boundary
convection pairing (Eq. bttp), the column-wise reduced Radau quadrature of the nonlinear
term (Eq. QuadNL, AlgFconv) and the Jacobian of Eq. JacobianLocal0-1.

For time node i (weight w_i = tau/2 omega_i), state (v^i, p^i), test (z, q), Gamma = Gamma_D:

  R_v^i[z] = sum_a K_ia (v^a, z) - phi_i(t_{n-1}^+) (v_{n-1}, z)
           + w_i { (nu grad v^i, grad z) - (p^i, div z) - (v^i (x) v^i, grad z) - (f^i, z)
                   - nu <d_n v^i, z> + <p^i n, z> - nu <v^i - g^i, d_n z>
                   + nu gamma1/h <v^i - g^i, z> + gamma2/h <(v^i - g^i).n, z.n>
                   + <((v^i.n)^+ - 2 (v^i.n)^-) v^i, z> + <(g^i.n)^- g^i, z> }
  R_p^i[q] = w_i { -(div v^i, q) + <(v^i - g^i).n, q> }

The pressure row is the paper's algebraic row (M (x) (B_h + G^p)) V (Eq. InAlgNS2), which makes
the Jacobian's pressure coupling symmetric (J^21 = J^12^T).  The Dirichlet data of the
pressure row (<g.n, q>) is kept for consistency; it vanishes for every bundled problem.
Vectors are laid out [V^1 .. V^{k+1} | P^1 .. P^{k+1}] with each V^a component-major.
"""
import numpy as np
import scipy.sparse as sp


def _pos(y):
    return 0.5 * (np.abs(y) + y)


def _neg(y):
    return 0.5 * (np.abs(y) - y)


class SlabLayout:
    def __init__(self, space, k):
        self.space, self.k = space, k
        self.Nv, self.Np = space.Nv, space.Np
        self.Nst = (k + 1) * (self.Nv + self.Np)

    def v(self, U, a):
        return U[a * self.Nv:(a + 1) * self.Nv]

    def p(self, U, a):
        o = (self.k + 1) * self.Nv
        return U[o + a * self.Np:o + (a + 1) * self.Np]

    def voff(self, a):
        return a * self.Nv

    def poff(self, a):
        return (self.k + 1) * self.Nv + a * self.Np


def velocity_at_qp(space, V):
    """Values [ncells, Q, d] and physical gradients [ncells, Q, d(comp), d(dir)] of a velocity field."""
    d = space.d
    loc = np.stack([V[space.cell_nodes + c * space.nnodes] for c in range(d)], axis=1)  # [cells,d,nloc]
    val = np.einsum("qj,kcj->kqc", space.ref.phi, loc)
    grad = np.einsum("kqjl,kcj->kqcl", space.gphi, loc)
    return val, grad


def velocity_at_face(space, V, axis, side):
    d = space.d
    fd = space.face_data[(axis, side)]
    loc = np.stack([V[space.cell_nodes + c * space.nnodes] for c in range(d)], axis=1)
    val = np.einsum("pj,kcj->kpc", fd["phi"], loc)
    grad = np.einsum("kpjl,kcj->kpcl", fd["gphi"], loc)
    return val, grad


def pressure_at(space, P, psi):
    loc = P[space.cell_pdofs]                      # [cells, npc]
    return np.einsum("qm,km->kq", psi, loc)


# ----------------------------------------------------------------------------- residual
def residual(space, td, U, Vprev, prob, t0, gamma1=10.0, gamma2=10.0, bconv=True, hscale=None):
    """R_n(U; V_{n-1}) of Eq. InAlgNS (LHS minus RHS), FP64."""
    lay = SlabLayout(space, td.k)
    d, nu = space.d, prob.nu
    ref = space.ref
    R = np.zeros(lay.Nst)
    times = td.times(t0)
    Mv = mass_velocity(space)
    for i in range(td.k + 1):
        wi, ti = td.w[i], times[i]
        Rv = np.zeros((space.mesh.ncells, d, space.nloc))
        Rp = np.zeros((space.mesh.ncells, space.npc))
        V = lay.v(U, i)
        P = lay.p(U, i)
        v, gv = velocity_at_qp(space, V)
        p = pressure_at(space, P, ref.psi)
        f = prob.f(space.xq, ti)
        JxW = space.JxW
        # flux tested with grad z_c: nu grad v_c - p e_c - v_c v
        flux = nu * gv - p[..., None, None] * np.eye(d)[None, None] - v[..., :, None] * v[..., None, :]
        Rv += np.einsum("kq,kqcl,kqjl->kcj", JxW, flux, space.gphi)
        Rv -= np.einsum("kq,kqc,qj->kcj", JxW, f, ref.phi)
        div = np.einsum("kqcc->kq", gv)
        Rp -= np.einsum("kq,kq,qm->km", JxW, div, ref.psi)
        for axis in range(d):
            for side in (0, 1):
                cells = _boundary_cells(space, axis, side)
                fd = space.face_data[(axis, side)]
                vf, gvf = velocity_at_face(space, V, axis, side)
                pf = pressure_at(space, P, fd["psi"])
                g = prob.g(fd["x"], ti)
                nrm = fd["normal"]
                JxWf = fd["JxW"]
                h = nitsche_length(space, JxWf, hscale)
                dnv = np.einsum("kpcl,kpl->kpc", gvf, nrm)
                e = vf - g
                en = np.einsum("kpc,kpc->kp", e, nrm)
                y = np.einsum("kpc,kpc->kp", vf, nrm)
                gn = np.einsum("kpc,kpc->kp", g, nrm)
                val = (-nu * dnv + (nu * gamma1 / h)[:, None, None] * e
                       + (gamma2 / h)[:, None, None] * en[..., None] * nrm + pf[..., None] * nrm)
                if bconv:
                    val = val + (_pos(y) - 2.0 * _neg(y))[..., None] * vf + _neg(gn)[..., None] * g
                dnz = np.einsum("kpjl,kpl->kpj", fd["gphi"], nrm)
                contrib = np.einsum("kp,kpc,pj->kcj", JxWf, val, fd["phi"])
                contrib -= nu * np.einsum("kp,kpc,kpj->kcj", JxWf, e, dnz)
                Rv[cells] += contrib[cells]
                Rp[cells] += np.einsum("kp,kp,pm->km", JxWf, en, fd["psi"])[cells]
        # scatter spatial parts scaled by w_i
        Rvi = np.zeros(lay.Nv)
        for c in range(d):
            np.add.at(Rvi, space.cell_nodes + c * space.nnodes, Rv[:, c, :])
        Rpi = np.zeros(lay.Np)
        np.add.at(Rpi, space.cell_pdofs, Rp)
        R[lay.voff(i):lay.voff(i) + lay.Nv] += wi * Rvi
        R[lay.poff(i):lay.poff(i) + lay.Np] += wi * Rpi
        # temporal coupling (K (x) M_h) V and jump (C (x) M_h) V_{n-1}
        acc = np.zeros(lay.Nv)
        for a in range(td.k + 1):
            acc += td.K[i, a] * (Mv @ lay.v(U, a))
        acc -= td.C[i] * (Mv @ Vprev)
        R[lay.voff(i):lay.voff(i) + lay.Nv] += acc
    return R


def nitsche_length(space, face_JxW, hscale=None):
    """h_{Gamma_D} of Eq. def-b-gam-3 per cell for one face: h_F / (p (p+1)), p = r+1.

    `hscale` replaces the factor 1 / (p (p+1)); the multigrid levels pass the finest level's
    value times n_level / n_finest, so that every level keeps the finest level's penalty.

    h_F = |K| / |F| (cell volume over the area of this face).  The paper does not define
    h_{Gamma_D}.  With the plain h_F and gamma_1 = gamma_2 = 10 the discrete problem is not
    coercive for Q_{r+1} (the convergence test of Sec. 5.1 diverges for r = 3); the
    degree-scaled length is the usual interior-penalty scaling, and with it the oracle
    reproduces the errors printed in Table conv-ns.
    """
    p = space.r + 1
    if hscale is None:
        hscale = 1.0 / (p * (p + 1))
    return space.cell_volume / face_JxW.sum(axis=1) * hscale


def _boundary_cells(space, axis, side):
    n = space.mesh.n
    return np.nonzero(space.mesh.cell_multi[:, axis] == (0 if side == 0 else n - 1))[0]


# ----------------------------------------------------------------------------- element matrices
def element_matrices(space, V, nu, gamma1=10.0, gamma2=10.0, bconv=True, hscale=None):
    """Per-cell spatial matrices of one time node at velocity state V.

    Returns A [cells, d*nloc, d*nloc] = nu A_h + N^{b,r}(gamma) + H'(V) + N^c'(V) (velocity block,
    test row, trial column) and B [cells, npc, d*nloc] = B_h + G^p (Eq. DefMAB, DefNitscheSpatial1).
    Local velocity index = component * nloc + node.
    """
    d, nl = space.d, space.nloc
    ref = space.ref
    nc = space.mesh.ncells
    v, _ = velocity_at_qp(space, V)
    JxW, gphi, phi = space.JxW, space.gphi, ref.phi
    A = np.zeros((nc, d, nl, d, nl))
    lap = nu * np.einsum("kq,kqil,kqjl->kij", JxW, gphi, gphi)
    # convection -(dv (x) v + v (x) dv, grad z): test phi_i e_c, trial phi_j e_c'
    t1 = -np.einsum("kq,qj,kql,kqil->kij", JxW, phi, v, gphi)          # delta_cc' part
    t2 = -np.einsum("kq,kqc,qj,kqie->kciej", JxW, v, phi, gphi)        # v_c phi_j d_c' phi_i
    for c in range(d):
        A[:, c, :, c, :] += lap + t1
    A += t2
    B = -np.einsum("kq,qm,kqje->kmej", JxW, ref.psi, gphi)
    for axis in range(d):
        for side in (0, 1):
            cells = _boundary_cells(space, axis, side)
            fd = space.face_data[(axis, side)]
            JxWf, nrm, fphi, fgphi = fd["JxW"], fd["normal"], fd["phi"], fd["gphi"]
            h = nitsche_length(space, JxWf, hscale)
            vf, _ = velocity_at_face(space, V, axis, side)
            y = np.einsum("kpc,kpc->kp", vf, nrm)
            dn = np.einsum("kpjl,kpl->kpj", fgphi, nrm)
            Af = np.zeros((nc, d, nl, d, nl))
            scal = (-nu * np.einsum("kp,kpj,pi->kij", JxWf, dn, fphi)
                    - nu * np.einsum("kp,pj,kpi->kij", JxWf, fphi, dn)
                    + (nu * gamma1 / h)[:, None, None] * np.einsum("kp,pj,pi->kij", JxWf, fphi, fphi))
            if bconv:
                scal = scal + np.einsum("kp,kp,pj,pi->kij", JxWf, _pos(y) - 2.0 * _neg(y), fphi, fphi)
            for c in range(d):
                Af[:, c, :, c, :] += scal
            Af += (gamma2 / h)[:, None, None, None, None] * np.einsum(
                "kp,kpc,kpe,pi,pj->kciej", JxWf, nrm, nrm, fphi, fphi)
            if bconv:
                Af += np.einsum("kp,kp,kpe,kpc,pi,pj->kciej",
                                JxWf, 0.5 * (3.0 - np.sign(y)), nrm, vf, fphi, fphi)
            A[cells] += Af[cells]
            Bf = np.einsum("kp,pm,kpe,pj->kmej", JxWf, fd["psi"], nrm, fphi)
            B[cells] += Bf[cells]
    return A.reshape(nc, d * nl, d * nl), B.reshape(nc, space.npc, d * nl)


def element_mass(space):
    """Per-cell scalar velocity mass [cells, nloc, nloc] and pressure mass [cells, npc, npc]."""
    Mc = np.einsum("kq,qi,qj->kij", space.JxW, space.ref.phi, space.ref.phi)
    Mp = np.einsum("kq,qi,qj->kij", space.JxW, space.ref.psi, space.ref.psi)
    return Mc, Mp


def mass_velocity(space):
    """Global M_h for one vector velocity field (block diagonal over components)."""
    Mc, _ = element_mass(space)
    d = space.d
    rows, cols, vals = [], [], []
    for c in range(d):
        gi = space.cell_nodes + c * space.nnodes
        rows.append(np.repeat(gi, gi.shape[1], axis=1).ravel())
        cols.append(np.tile(gi, (1, gi.shape[1])).ravel())
        vals.append(Mc.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(space.Nv, space.Nv))


def mass_pressure(space):
    _, Mp = element_mass(space)
    gi = space.cell_pdofs
    n = gi.shape[1]
    return sp.csr_matrix((Mp.ravel(), (np.repeat(gi, n, axis=1).ravel(), np.tile(gi, (1, n)).ravel())),
                         shape=(space.Np, space.Np))


def _scatter_block(rows_idx, cols_idx, blocks):
    n1, n2 = rows_idx.shape[1], cols_idx.shape[1]
    r = np.repeat(rows_idx, n2, axis=1).ravel()
    c = np.tile(cols_idx, (1, n1)).ravel()
    return r, c, blocks.ravel()


def jacobian(space, td, U, nu, gamma1=10.0, gamma2=10.0, bconv=True, vstar=None, hscale=None):
    """Assembled slab Jacobian J_n(U) (Eq. JacobianLocal0-1) as a CSR matrix.

    With `vstar` given, every time node's convection Jacobian is evaluated at the single
    velocity field vstar instead of V^a: the midpoint surrogate of Eq. DefTildeHn.
    """
    lay = SlabLayout(space, td.k)
    rows, cols, vals = [], [], []
    Mv = mass_velocity(space).tocoo()
    for i in range(td.k + 1):
        for a in range(td.k + 1):
            if td.K[i, a] != 0.0:
                rows.append(Mv.row + lay.voff(i))
                cols.append(Mv.col + lay.voff(a))
                vals.append(td.K[i, a] * Mv.data)
        Vs = lay.v(U, i) if vstar is None else vstar
        A, B = element_matrices(space, Vs, nu, gamma1, gamma2, bconv, hscale)
        wi = td.w[i]
        vd = space.cell_vdofs
        pd = space.cell_pdofs
        r, c, v = _scatter_block(vd + lay.voff(i), vd + lay.voff(i), wi * A)
        rows.append(r); cols.append(c); vals.append(v)
        r, c, v = _scatter_block(pd + lay.poff(i), vd + lay.voff(i), wi * B)
        rows.append(r); cols.append(c); vals.append(v)
        r, c, v = _scatter_block(vd + lay.voff(i), pd + lay.poff(i), wi * np.transpose(B, (0, 2, 1)))
        rows.append(r); cols.append(c); vals.append(v)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(lay.Nst, lay.Nst))


def apply(space, td, U, x, nu, gamma1=10.0, gamma2=10.0, bconv=True):
    """y = J_n(U) x through the assembled Jacobian (the plain definition of the operator apply)."""
    return jacobian(space, td, U, nu, gamma1, gamma2, bconv) @ x


def slab_mass(space, td):
    """Block-diagonal mass of the norm || . ||_M: diag(M^tau (x) M_h, M^tau (x) M_h^p) (Sec. 4.1)."""
    Mv = mass_velocity(space)
    Mp = mass_pressure(space)
    blocks = [td.w[a] * Mv for a in range(td.k + 1)] + [td.w[a] * Mp for a in range(td.k + 1)]
    return sp.block_diag(blocks, format="csr")


def mnorm(space, td, Z, Mslab=None):
    M = slab_mass(space, td) if Mslab is None else Mslab
    return float(np.sqrt(max(Z @ (M @ Z), 0.0)))


def interpolate_velocity(space, func):
    """Nodal interpolation of a vector field at the GLL nodes (reading of v_{0,h} in Problem 2.1)."""
    X = space.node_coords()
    vals = func(X)
    return np.concatenate([vals[:, c] for c in range(space.d)])
