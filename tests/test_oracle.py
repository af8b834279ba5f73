"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests calls the CUDA library.  Each pin checks the oracle
against something other than itself: closed forms of the lemmas, a textbook
FD convergence order, a brute-force dense pseudoinverse, a sparse direct
solve, CG's finite-termination property, or values printed in the paper.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Sec. 3.1/3.2
@pytest.mark.parametrize("bc", o.BCS)
@pytest.mark.parametrize("n", [3, 4, 5, 7, 8, 33, 64, 65])
def test_lemma_spectra_match_lap1d(bc, n):
    """Lemmas spectrumP/D/N/M: closed-form pairs are eigenpairs of eq. (lap1d)."""
    lam, V = o.spectrum_closed_form(n, bc)
    L = o.lap1d(n, bc)
    assert V.shape == (n, n)
    assert np.abs(L @ V - V * lam).max() <= 1e-12
    assert np.abs(np.sort(lam) - np.linalg.eigvalsh(L)).max() <= 1e-12
    # eigenvalues lie in [0, 4]; zero only for P and N (discussion after the lemmas)
    assert lam.min() >= -1e-14 and lam.max() <= 4 + 1e-14
    assert (np.abs(lam).min() < 1e-14) == (bc in ("P", "N"))


@pytest.mark.parametrize("bc", o.BCS)
def test_lap1d_symmetric_and_nullspace(bc):
    L = o.lap1d(9, bc)
    assert np.array_equal(L, L.T)
    null = np.abs(L @ np.ones(9)).max() == 0.0
    assert null == (bc in ("P", "N"))


def test_lap1d_spacing_scales_operator():
    assert np.allclose(o.lap1d(6, "D", 0.5), 4.0 * o.lap1d(6, "D"))


# ---------------------------------------------------------------- Sec. 3.3
def _grid_and_solution(bc, n):
    """Grid points, spacing and a smooth manufactured u with -u'' = k2 u on [0, 1] obeying bc."""
    j = np.arange(1, n + 1, dtype=np.float64)
    if bc == "D":
        h = 1.0 / (n + 1); x = j * h
        return h, np.sin(math.pi * x), math.pi ** 2
    if bc == "P":
        h = 1.0 / n; x = j * h
        return h, np.sin(2 * math.pi * x) + np.cos(2 * math.pi * x), 4 * math.pi ** 2
    if bc == "N":
        h = 1.0 / n; x = (j - 0.5) * h
        return h, np.cos(math.pi * x), math.pi ** 2
    if bc == "DN":
        h = 1.0 / (n + 0.5); x = j * h
        return h, np.sin(0.5 * math.pi * x), 0.25 * math.pi ** 2
    if bc == "ND":
        h = 1.0 / (n + 0.5); x = (j - 0.5) * h
        return h, np.cos(0.5 * math.pi * x), 0.25 * math.pi ** 2
    raise ValueError(bc)


def _fd_error(bcs, n):
    shape = (n, n, 1)
    hx, ux, kx = _grid_and_solution(bcs[0], n)
    hy, uy, ky = _grid_and_solution(bcs[1], n)
    u = ux[:, None, None] * uy[None, :, None]
    f = (kx + ky) * u
    res = o.pcg(shape, (bcs[0], bcs[1], None), (hx, hy, 1.0), f, tol=1e-13, maxit=20)
    return np.abs(res.U - u).max()


@pytest.mark.parametrize("bcs", [("D", "D"), ("P", "N"), ("N", "N"), ("DN", "P"), ("ND", "D"), ("P", "P")])
def test_textbook_second_order_convergence(bcs):
    """The FD solution of -Laplace(u) = f converges as O(h^2) to a smooth u: pins the sign, the 1/h^2
    scaling, each corner of eq. (lap1d) and the Kronecker assembly of eq. (ourproblem2)."""
    e1 = _fd_error(bcs, 12)
    e2 = _fd_error(bcs, 24)
    assert e2 < 0.05
    assert 3.0 < e1 / e2 < 5.0, (e1, e2)


def test_textbook_convergence_3d():
    def err(n):
        hx, ux, kx = _grid_and_solution("P", n)
        hy, uy, ky = _grid_and_solution("D", n)
        hz, uz, kz = _grid_and_solution("ND", n)
        u = ux[:, None, None] * uy[None, :, None] * uz[None, None, :]
        res = o.pcg((n, n, n), ("P", "D", "ND"), (hx, hy, hz), (kx + ky + kz) * u, tol=1e-13)
        return np.abs(res.U - u).max()

    e1, e2 = err(8), err(16)
    assert 3.0 < e1 / e2 < 5.0, (e1, e2)


SMALL_SHAPES = [(3, 4, 5), (6, 5, 4), (4, 3, 1), (5, 7, 1)]


@pytest.mark.parametrize("shape", SMALL_SHAPES)
@pytest.mark.parametrize("bcs", [("P", "N", "P"), ("D", "DN", "ND"), ("N", "N", "N"), ("P", "D", "N")])
def test_kron_sum_spectrum_is_all_eigenvalue_sums(shape, bcs):
    """sigma(L_3D) = {lambda_i + lambda_j + lambda_k} with the closed-form 1D spectra (Sec. 3.3)."""
    L = o.kron_sum(shape, bcs).toarray()
    assert np.array_equal(L, L.T)
    lam = [o.spectrum_closed_form(ell, bc)[0] if ell > 1 else np.zeros(1) for ell, bc in zip(shape, bcs)]
    sums = np.sort((lam[0][:, None, None] + lam[1][None, :, None] + lam[2][None, None, :]).ravel())
    assert np.abs(np.sort(np.linalg.eigvalsh(L)) - sums).max() < 1e-12
    singular = np.abs(L @ np.ones(L.shape[0])).max() == 0.0
    assert singular == o.is_singular(shape, bcs)


@pytest.mark.parametrize("bcs", list(itertools.product(o.BCS, repeat=3))[::7])
def test_assembled_operator_equals_mode_product_form(bcs):
    """vec(L_n x1 U + L_q x2 U + L_t x3 U) = L_3D vec(U): eq. (ourproblem) vs eq. (ourproblem2)."""
    shape = (5, 4, 3)
    U = np.random.default_rng(1).standard_normal(shape)
    Ls = o.axis_matrices(shape, bcs, (1.0, 0.7, 1.3))
    a = o.vec(o.apply_minus_laplacian(U, Ls))
    b = o.kron_sum(shape, bcs, (1.0, 0.7, 1.3)) @ o.vec(U)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_vec_order_is_first_index_fastest():
    U = np.arange(24).reshape((2, 3, 4), order="F")
    assert list(o.vec(U)[:4]) == [U[0, 0, 0], U[1, 0, 0], U[0, 1, 0], U[1, 1, 0]]


# ---------------------------------------------------------------- Sec. 4.3.3
@pytest.mark.parametrize("shape", SMALL_SHAPES + [(8, 6, 5)])
@pytest.mark.parametrize("bcs", [("P", "N", "P"), ("D", "DN", "ND"), ("N", "N", "N"), ("P", "P", "D"), ("ND", "N", "P")])
def test_pinv_apply_equals_dense_pseudoinverse(shape, bcs):
    """Algorithm 7 with Algorithm 5's G equals the brute-force dense pseudoinverse L^+ r."""
    r = np.random.default_rng(2).standard_normal(shape)
    Vs, lams, G = o.pinv_init(shape, bcs)
    z = o.pinv_apply(r, Vs, G)
    ref = o.minnorm_dense(shape, bcs, (1.0, 1.0, 1.0), r)
    assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()
    # exactly one zeroed eigenvalue sum when singular, none otherwise
    assert int((G == 0).sum()) == (1 if o.is_singular(shape, bcs) else 0)


def test_pinv_with_spacing_matches_sparse_solve():
    shape, bcs, hs = (9, 7, 6), ("D", "ND", "DN"), (0.5, 1.5, 2.0)
    r = np.random.default_rng(3).standard_normal(shape)
    Vs, _, G = o.pinv_init(shape, bcs, hs)
    z = o.pinv_apply(r, Vs, G)
    ref = o.solve_sparse_direct(shape, bcs, hs, r)
    assert np.abs(z - ref).max() <= 1e-11 * np.abs(ref).max()


def test_pinv_threshold_matches_numerical_zero_eigenvalues():
    """Reading of the 1e-13 threshold: 1D P/N zero eigenvalues from eigh are far below it,
    the smallest nonzero sums far above it."""
    for n in (3, 64, 256, 1000):
        for bc in ("P", "N"):
            lam = np.linalg.eigvalsh(o.lap1d(n, bc))
            assert abs(lam[0]) < 1e-13 * 0.1
            assert lam[1] > 1e-6


# ---------------------------------------------------------------- Algorithm 1
@pytest.mark.parametrize("bcs", [("P", "P", "N"), ("D", "D", "D"), ("P", "D", "DN"), ("N", "ND", "P")])
def test_manufactured_eigenvector_solution(bcs):
    """U = v_i (x) v_j (x) v_k from the lemmas gives H = (lam_i+lam_j+lam_k) U exactly."""
    shape = (8, 6, 5)
    lv = [o.spectrum_closed_form(ell, bc) for ell, bc in zip(shape, bcs)]
    i, j, k = 3, 2, 1
    U = lv[0][1][:, i][:, None, None] * lv[1][1][:, j][None, :, None] * lv[2][1][:, k][None, None, :]
    H = (lv[0][0][i] + lv[1][0][j] + lv[2][0][k]) * U
    res = o.pcg(shape, bcs, (1.0, 1.0, 1.0), H, tol=1e-14, maxit=10)
    assert np.abs(res.U - U).max() <= 1e-12 * np.abs(U).max()


@pytest.mark.parametrize("bcs", [("P", "P", "N"), ("D", "N", "DN")])
def test_one_step_exactness(bcs):
    """With U0 = 0 and M = L^+, Z0 = L^+ H is the solution: alpha_1 = 1 and U_1 = M(H)."""
    shape = (10, 8, 6)
    H = np.random.default_rng(4).standard_normal(shape)
    res = o.pcg(shape, bcs, (1.0, 1.0, 1.0), H, tol=1e-15, maxit=3)
    assert abs(res.alphas[0] - 1.0) < 1e-12
    assert res.true_res[1] < 1e-13
    Vs, _, G = o.pinv_init(shape, bcs)
    singular = o.is_singular(shape, bcs)
    Hc = o.center(H) if singular else H
    Z0 = o.pinv_apply(Hc, Vs, G)
    if singular:
        Z0 = o.center(Z0)
    assert np.abs(res.U - Z0).max() < 1e-12 * np.abs(Z0).max()


def test_pcg_matches_sparse_direct_nonsingular():
    shape, bcs = (16, 12, 10), ("D", "P", "ND")
    H = np.random.default_rng(5).standard_normal(shape)
    res = o.pcg(shape, bcs, (1.0, 1.0, 1.0), H, tol=1e-13)
    ref = o.solve_sparse_direct(shape, bcs, (1.0, 1.0, 1.0), H)
    assert np.abs(res.U - ref).max() <= 1e-11 * np.abs(ref).max()
    assert res.iters <= 3  # "two or three are sufficient" (Sec. 6)


def test_pcg_singular_is_minimum_norm_and_zero_mean():
    shape, bcs = (7, 6, 5), ("P", "N", "P")
    H = np.random.default_rng(6).standard_normal(shape) + 0.3  # nonzero mean gets projected out
    res = o.pcg(shape, bcs, (1.0, 1.0, 1.0), H, tol=1e-13)
    assert abs(res.U.mean()) < 1e-15 * np.abs(res.U).max() * res.U.size
    ref = o.minnorm_dense(shape, bcs, (1.0, 1.0, 1.0), o.center(H))
    assert np.abs(res.U - ref).max() <= 1e-11 * np.abs(ref).max()
    assert abs(res.removed_mean - H.mean()) < 1e-15


def test_plain_cg_finite_termination():
    """Algorithm 1 with M = I terminates in at most (#distinct eigenvalues) steps: a dropped
    beta or a wrong alpha would not."""
    shape, bcs = (5, 3, 1), ("D", "D", None)
    lam = [o.spectrum_closed_form(5, "D")[0], o.spectrum_closed_form(3, "D")[0]]
    distinct = len(np.unique(np.round((lam[0][:, None] + lam[1][None, :]).ravel(), 10)))
    H = np.random.default_rng(7).standard_normal(shape)
    res = o.pcg(shape, ("D", "D", "D"), (1.0, 1.0, 1.0), H, tol=1e-11, maxit=200, precond="none")
    assert res.true_res[-1] <= 1e-11
    assert res.iters <= distinct


def test_warm_start_converges_to_same_solution():
    shape, bcs = (9, 8, 7), ("P", "P", "N")
    H = np.random.default_rng(8).standard_normal(shape)
    U0 = np.random.default_rng(9).standard_normal(shape)
    a = o.pcg(shape, bcs, (1.0, 1.0, 1.0), H, tol=1e-13)
    b = o.pcg(shape, bcs, (1.0, 1.0, 1.0), H, U0=U0, tol=1e-13)
    assert np.abs(a.U - b.U).max() < 1e-11 * np.abs(a.U).max()


# ---------------------------------------------------------------- Sec. 3.4.2
def test_rhs_bc_update_problem2_reading():
    """Problem 2: u = 0 on the left (D), outward derivative -1/2 on the right (N), periodic
    vertically, no charge: the potential falls linearly with slope -1/2 (Sec. 5.3)."""
    n, q, h = 40, 12, 0.25
    H = np.zeros((n, q, 1))
    H = o.rhs_add_bc(H, ("DN", "P", None), (h, 1.0, 1.0), [0.0, -0.5, 0, 0, 0, 0])
    res = o.pcg((n, q, 1), ("DN", "P", None), (h, 1.0, 1.0), H, tol=1e-14)
    x = np.arange(1, n + 1) * h
    assert np.abs(res.U[:, :, 0] - (-0.5 * x)[:, None]).max() < 1e-10


def test_rhs_bc_update_dirichlet_both_ends():
    n = 9
    H = o.rhs_add_bc(np.zeros((n, 3, 1)), ("D", "P", None), (1.0, 1.0, 1.0), [1.0, 3.0, 0, 0, 0, 0])
    res = o.pcg((n, 3, 1), ("D", "P", None), (1.0, 1.0, 1.0), H, tol=1e-14)
    j = np.arange(1, n + 1)
    assert np.abs(res.U[:, 0, 0] - (1.0 + 2.0 * j / (n + 1))).max() < 1e-12


# ---------------------------------------------------------------- Sec. 5.2
def test_normalization_values_from_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "normalization.txt")) if l.strip() and l[0] != "#"]
    for n, q, t, expect in rows:
        H = np.random.default_rng(10).standard_normal((int(n), int(q), int(t)))
        assert abs(np.linalg.norm(o.normalize_rhs(H).ravel()) - float(expect)) <= 1e-15 * float(expect) * 10


def test_cost_model_counts_mode_products():
    """Table PInvPcost: two passes of three mode products (2 flops per multiply-add) and one
    Hadamard product give 4nqt(n+q+t+1/4)."""
    n, q, t = 256, 256, 128
    per_direction = 2 * n * q * t * n + 2 * n * q * t * q + 2 * n * q * t * t
    assert o.pinv_apply_flops(n, q, t) == 2 * per_direction + n * q * t


# ---------------------------------------------------------------- Sec. 2: field from potential
def test_efield_periodic_sine_is_exact_discrete_cosine():
    """Central difference of sin(2 pi j / n) is cos(2 pi j / n) sin(2 pi / n) / h exactly."""
    n, q, t, h = 24, 5, 4, 0.5
    j = np.arange(n)
    U = np.sin(2 * np.pi * j / n)[:, None, None] * np.ones((n, q, t))
    ex, ey, ez = o.efield(U, ("P", "N", "D"), (h, 1.0, 1.0))
    want = -np.cos(2 * np.pi * j / n) * np.sin(2 * np.pi / n) / h
    assert np.abs(ex - want[:, None, None]).max() < 1e-14
    assert np.abs(ey).max() == 0.0  # U constant in y: Neumann ghosts mirror it


@pytest.mark.parametrize("bc", ["D", "N", "DN", "ND"])
def test_efield_linear_potential_with_consistent_face_data(bc):
    """u = c + a x h on x = -1..n: with face data taken from u itself the field is -a everywhere."""
    n, h, a, c = 9, 0.25, 1.7, -0.3
    x = np.arange(n)
    U = (c + a * x * h)[:, None, None] * np.ones((n, 3, 1))
    sk, ek = {"D": ("D", "D"), "N": ("N", "N"), "DN": ("D", "N"), "ND": ("N", "D")}[bc]
    start = c - a * h if sk == "D" else -a        # Dirichlet value at the ghost, or outward derivative (-x)
    end = c + a * n * h if ek == "D" else a       # Dirichlet value at the ghost, or outward derivative (+x)
    ex, ey = o.efield(U, (bc, "P", "P"), (h, 1.0, 1.0), bvals=[start, end, 0, 0, 0, 0])
    assert np.abs(ex + a).max() < 1e-12
    assert np.abs(ey).max() == 0.0


def test_efield_second_order_against_analytic_gradient():
    """Smooth periodic potential: the discrete field converges at second order."""
    errs = []
    for n in (16, 32, 64):
        h = 2 * np.pi / n
        xs = np.arange(n) * h
        U = (np.sin(xs)[:, None] * np.cos(2 * xs)[None, :])[:, :, None]
        ex, ey = o.efield(U, ("P", "P", "P"), (h, h, 1.0))
        gx = -(np.cos(xs)[:, None] * np.cos(2 * xs)[None, :])[:, :, None]
        gy = (2 * np.sin(xs)[:, None] * np.sin(2 * xs)[None, :])[:, :, None]
        errs.append(max(np.abs(ex - gx).max(), np.abs(ey - gy).max()))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


# ---------------------------------------------------------------- Sec. 4.3.1: Jacobi(p, omega)
def test_jacobi_one_step_is_scaled_residual():
    """p = 1: Z = R / (omega * (diag L_n + diag L_q + diag L_t)), the corner entries included."""
    shape, bcs, hs, om = (6, 5, 4), ("DN", "N", "P"), (0.5, 1.0, 2.0), 1.3
    R = np.random.default_rng(3).standard_normal(shape)
    Os, Dinv = o.jacobi_init(shape, bcs, hs, om)
    d = np.diag(o.kron_sum(shape, bcs, hs).toarray())
    want = o.unvec(o.vec(R) / (om * d), shape)
    assert np.abs(o.jacobi_apply(R, Os, Dinv, 1) - want).max() < 1e-15 * np.abs(want).max()


def test_jacobi_many_steps_converge_to_the_inverse():
    """As p grows the stationary iteration from 0 converges to L^-1 R (nonsingular operator)."""
    shape, bcs, hs = (5, 4, 3), ("D", "DN", "ND"), (1.0, 1.0, 1.0)
    R = np.random.default_rng(4).standard_normal(shape)
    Os, Dinv = o.jacobi_init(shape, bcs, hs, 1.3)
    Z = o.jacobi_apply(R, Os, Dinv, 3000)
    x = o.solve_sparse_direct(shape, bcs, hs, R)
    assert np.abs(Z - x).max() < 1e-10 * np.abs(x).max()


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_jacobi_preconditioner_is_symmetric(p):
    """<M a, b> = <a, M b>: a dropped or transposed O_omega would break it."""
    shape, bcs, hs = (6, 5, 4), ("P", "ND", "N"), (0.7, 1.0, 1.3)
    rng = np.random.default_rng(5)
    a, b = rng.standard_normal(shape), rng.standard_normal(shape)
    Os, Dinv = o.jacobi_init(shape, bcs, hs, 1.3)
    lhs = np.vdot(o.jacobi_apply(a, Os, Dinv, p), b)
    rhs = np.vdot(a, o.jacobi_apply(b, Os, Dinv, p))
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)


def test_comparator_ordering_on_a_small_problem():
    """Experiment 2's qualitative ordering: p-inv needs the fewest iterations, then Jacobi(3, 1.3), then CG."""
    shape, bcs = (24, 16, 1), ("P", "P", None)
    H = o.normalize_rhs(o.center(np.random.default_rng(6).standard_normal(shape)))
    it = {k: o.pcg(shape, bcs, (1, 1, 1), H, tol=1e-10, maxit=2000, precond=k).iters
          for k in ("pinv", "jacobi", "none")}
    assert it["pinv"] < it["jacobi"] < it["none"]
