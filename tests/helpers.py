"""Shared test helpers: oracle set-up from the same seeded inputs, GPU availability, and the
5^d-cell sub-block used to check full-size GPU results against the oracle cell by cell."""
import itertools

import numpy as np

from oracle import forms
from oracle.mesh import Mesh, Space
from oracle.reference import TimeData
from paper_2602_13841_gb300 import inputs


def oracle_space(d, n, r, verts):
    return Space(Mesh(d, n, verts), r)


def have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def build_and_load():
    from paper_2602_13841_gb300 import build, stmg
    build.build()
    return stmg.load()


class Block:
    """The 5^d block of cells around `cell` (shifted inside the domain), with index maps
    from block numbering to the big mesh.  The block's artificial boundary faces carry Nitsche
    terms; the symmetric term -nu <v, d_n z> reaches every node of a block-boundary cell, so
    the sample cell keeps one cell of distance from them and its rows are exact."""

    W = 5

    def __init__(self, d, n, r, k, verts_big, cell):
        W = self.W
        assert n >= W
        self.d, self.n, self.r, self.k = d, n, r, k
        self.s = [min(max(c - 2, 0), n - W) for c in cell]
        self.pos = [c - s for c, s in zip(cell, self.s)]
        self.cell = cell
        Vb = verts_big.reshape(*([n + 1] * d)[::-1], d)    # [z][y][x][d]
        sl = tuple(slice(s, s + W + 1) for s in self.s[::-1])
        self.verts = Vb[sl].reshape(-1, d)
        self.space = oracle_space(d, W, r, self.verts)
        N1b, N1 = W * (r + 1) + 1, (r + 1) * n + 1
        self.N1, self.N1b = N1, N1b
        nodes = np.array(list(itertools.product(*([range(N1b)] * d))))[:, ::-1]
        gm = nodes + (r + 1) * np.array(self.s)
        self.node_map = np.einsum("il,l->i", gm, N1 ** np.arange(d))
        cells = np.array(list(itertools.product(*([range(W)] * d))))[:, ::-1]
        self.cell_map = np.einsum("il,l->i", cells + np.array(self.s), n ** np.arange(d))
        self.npc = self.space.npc
        nn_big = N1 ** d
        self.Nv_big, self.Np_big = d * nn_big, n ** d * self.npc
        # block slab vector index -> big slab vector index
        idx = []
        for a in range(k + 1):
            for c in range(d):
                idx.append(a * self.Nv_big + c * nn_big + self.node_map)
        for a in range(k + 1):
            pc = (self.cell_map[:, None] * self.npc + np.arange(self.npc)[None, :]).ravel()
            idx.append((k + 1) * self.Nv_big + a * self.Np_big + pc)
        self.slab_map = np.concatenate(idx)
        self.vel_map = np.concatenate([c * nn_big + self.node_map for c in range(d)])
        # rows of the sample cell inside the block slab vector
        lay = forms.SlabLayout(self.space, k)
        bcell = int(np.dot(self.pos, W ** np.arange(d)))
        rows = []
        for a in range(k + 1):
            rows.append(lay.voff(a) + self.space.cell_vdofs[bcell])
        for a in range(k + 1):
            rows.append(lay.poff(a) + self.space.cell_pdofs[bcell])
        self.rows = np.concatenate(rows)


def seeded_state(n, seed):
    return inputs.uniform(n, seed)
