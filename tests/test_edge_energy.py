"""The edge form of <L p, p> that the mixed-form direction kernel sums.

The kernel never forms W = L P for the line-search denominator <W, P>
(Algorithm 1): it sums, per axis, the squared differences of P across the
edges of the grid -- each point's difference to its start-side neighbour (the
ghost value at the first point: wrapped for P, 0 for a Dirichlet start, the
point itself for a Neumann start) plus, at the last point of an axis whose end
is not periodic, the difference to the end ghost (0 for Dirichlet, the point
itself for Neumann).  Summation by parts on eq. (lap1d) says this equals
<L_3D vec P, vec P>; these CPU tests check it exactly on integer fields
against the oracle's assembled operator, for every boundary combination.
"""
import itertools

import numpy as np
import pytest

import oracle as o


def _start_ghost(p, bc):
    if bc == "P":
        return p[-1]
    if bc in ("D", "DN"):
        return np.zeros_like(p[0])
    return p[0]  # N, ND


def _end_ghost(p, bc):
    if bc in ("D", "ND"):
        return np.zeros_like(p[-1])
    return p[-1]  # N, DN (P is not counted at the end)


def edge_energy(P, bcs, ih2):
    """Per-axis sums of squared edge differences, weighted by 1/h^2, in exact integers."""
    total = 0
    for m in range(3):
        if P.shape[m] == 1:
            continue
        p = np.moveaxis(P, m, 0).astype(object)
        left = np.concatenate([_start_ghost(p, bcs[m])[None], p[:-1]], axis=0)
        s = ((p - left) ** 2).sum()
        if bcs[m] != "P":
            s += ((p[-1] - _end_ghost(p, bcs[m])) ** 2).sum()
        total += ih2[m] * s
    return total


@pytest.mark.parametrize("bcs", list(itertools.product(o.BCS, repeat=3)))
def test_edge_form_equals_quadratic_form_3d(bcs):
    shape = (5, 4, 3)
    rng = np.random.default_rng(hash(bcs) % 2**32)
    P = rng.integers(-1000, 1001, size=shape)
    L = o.kron_sum(shape, bcs)
    x = o.vec(P.astype(np.float64))
    quad = int(round(float(x @ (L @ x))))
    assert edge_energy(P, bcs, (1, 1, 1)) == quad


@pytest.mark.parametrize("bcs", list(itertools.product(o.BCS, repeat=2)))
def test_edge_form_equals_quadratic_form_2d_weighted(bcs):
    shape = (6, 5, 1)
    full = (bcs[0], bcs[1], "N")
    rng = np.random.default_rng(7)
    P = rng.integers(-50, 51, size=shape)
    ih2 = (4, 9, 0)  # h = 1/2, 1/3
    L = o.kron_sum(shape, full, (0.5, 1.0 / 3.0, 1.0))
    x = o.vec(P.astype(np.float64))
    quad = float(x @ (L @ x))
    assert abs(edge_energy(P, full, ih2) - quad) <= 1e-9 * max(1.0, abs(quad))


def test_edge_form_is_positive_for_nonconstant_fields():
    """Every term is non-negative; the sum vanishes only on the null space (constants for P/N)."""
    P = np.ones((4, 4, 4), dtype=np.int64) * 7
    assert edge_energy(P, ("P", "N", "P"), (1, 1, 1)) == 0
    assert edge_energy(P, ("P", "N", "D"), (1, 1, 1)) > 0
