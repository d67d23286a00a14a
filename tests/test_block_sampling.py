"""The 5^d-block sampling used by the full-size GPU parity tests is exact: on a mesh the
oracle can assemble whole, the block's rows of J x and R equal the full mesh's rows."""
import numpy as np
import pytest

from oracle import forms, problems
from oracle.mesh import Mesh, Space
from oracle.reference import TimeData
from paper_2602_13841_gb300 import inputs
from tests.helpers import Block


@pytest.mark.parametrize("d,n,r,k", [(2, 7, 2, 2), (3, 5, 1, 1)])
def test_block_rows_equal_full_rows(d, n, r, k):
    verts = inputs.vertices(d, n, 0.1, 5)
    sp = Space(Mesh(d, n, verts), r)
    td = TimeData(k, 0.05)
    lay = forms.SlabLayout(sp, k)
    U, x, Vp = inputs.uniform(lay.Nst, 1), inputs.uniform(lay.Nst, 2), inputs.uniform(lay.Nv, 3)
    prob = problems.make("TG2D" if d == 2 else "MMS3D", 1e-2)
    y = forms.jacobian(sp, td, U, 1e-2) @ x
    R = forms.residual(sp, td, U, Vp, prob, 0.2)
    cells = [[0] * d, [n - 1] * d, [1] + [n - 1] * (d - 1), [n // 2] * d]
    for cell in cells:
        B = Block(d, n, r, k, verts, cell)
        yb = forms.jacobian(B.space, td, U[B.slab_map], 1e-2) @ x[B.slab_map]
        assert np.abs(yb[B.rows] - y[B.slab_map[B.rows]]).max() < 1e-13 * np.abs(y).max()
        Rb = forms.residual(B.space, td, U[B.slab_map], Vp[B.vel_map], prob, 0.2)
        assert np.abs(Rb[B.rows] - R[B.slab_map[B.rows]]).max() < 1e-13 * np.abs(R).max()
