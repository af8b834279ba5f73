"""Plain CPU FP64 oracle for pseudoinverse-preconditioned CG on the FD Poisson problem.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code, tables or helpers with the CUDA library: every
quantity here is recomputed from the paper's definitions with numpy/scipy.

Index convention (the paper's, Sec. 2.1): a 3D array ``U`` has shape
``(n, q, t)`` with entries ``u[i, j, k]``; ``vec(U)`` stacks the first index
fastest, i.e. ``U.ravel(order="F")``.  A 2D problem is the 3D problem with
``t = 1`` and the third 1D operator equal to the 1x1 zero matrix, so that the
Kronecker sum of eq. (ourproblem2) reduces to its 2D form.

Contents, each citing the passage it follows:
  corners, lap1d          -- eq. (lap1d), Sec. 3.1
  spectrum_closed_form    -- Lemmas spectrumP / spectrumD / spectrumN / spectrumM, Sec. 3.2
  kron_sum                -- eq. (ourproblem2), Sec. 3.3
  apply_minus_laplacian   -- eq. (ourproblem), Sec. 3.3 (mode-product form)
  center                  -- eq. (centering), Sec. 3.4.1
  rhs_add_bc              -- Sec. 3.4.2
  efield                  -- Sec. 2 (field from potential), ghosts of eq. (lap1d) / Sec. 3.4.2
  pinv_init               -- Algorithms 4/5 (MPPI init), Sec. 4.3.3, threshold 1e-13
  pinv_apply              -- Algorithms 6/7 (MPPI apply), Sec. 4.3.3
  jacobi_init/apply       -- Algorithms 2/3, Sec. 4.3.1 (p steps of (weighted) Jacobi)
  pcg                     -- Algorithm 1 with Remark (orthogonality) centring of Z
  minnorm_dense           -- brute force: dense eigendecomposition of the assembled operator
  normalize_rhs           -- eq. (normalization), Sec. 5.2

Readings of places where the paper is silent:
  * grid spacing: the paper has unit spacing; a spacing h divides L_l by h^2;
  * threshold: |eigenvalue sum| < 1e-13 * max_l(1/h_l^2) counts as zero;
  * stopping: true relative residual ||H - L U|| / ||H|| <= tol (H centred);
  * centring: Z every iteration (Remark orthogonality), U once at exit;
  * field: the text writes the field as minus "nabla dot" of the scalar
    potential; read as the gradient, discretised by central differences with
    the Laplacian's ghost values at the faces.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

BCS = ("P", "D", "N", "DN", "ND")
PINV_THRESHOLD = 1e-13


# --------------------------------------------------------------------------
# Sec. 3.1, eq. (lap1d): the 1D FD minus-Laplacian and its corner entries
# --------------------------------------------------------------------------
def corners(bc: str) -> tuple[float, float, float]:
    """(alpha, beta, gamma) of L_n(alpha, beta, gamma) for a BC (list under eq. lap1d)."""
    table = {
        "P": (2.0, 2.0, -1.0),
        "D": (2.0, 2.0, 0.0),
        "N": (1.0, 1.0, 0.0),
        "DN": (2.0, 1.0, 0.0),
        "ND": (1.0, 2.0, 0.0),
    }
    if bc not in table:
        raise ValueError(f"unknown boundary condition {bc!r}")
    return table[bc]


def lap1d(n: int, bc: str | None, h: float = 1.0) -> np.ndarray:
    """Dense L_n(alpha, beta, gamma) / h^2 (eq. lap1d).  n >= 3.

    ``bc=None`` with ``n == 1`` is the absent axis of a 2D problem: the 1x1
    zero matrix.
    """
    if bc is None:
        if n != 1:
            raise ValueError("absent axis must have length 1")
        return np.zeros((1, 1))
    if n < 3:
        raise ValueError("eq. (lap1d) requires n >= 3")
    alpha, beta, gamma = corners(bc)
    L = np.zeros((n, n))
    for i in range(n):
        L[i, i] = 2.0
        if i > 0:
            L[i, i - 1] = -1.0
        if i < n - 1:
            L[i, i + 1] = -1.0
    L[0, 0] = alpha
    L[n - 1, n - 1] = beta
    L[0, n - 1] += gamma
    L[n - 1, 0] += gamma
    return L / (h * h)


# --------------------------------------------------------------------------
# Sec. 3.2, Lemmas spectrumP/D/N/M: closed-form eigenpairs (not normalised)
# --------------------------------------------------------------------------
def spectrum_closed_form(n: int, bc: str) -> tuple[np.ndarray, np.ndarray]:
    """Eigenvalues and (unnormalised) eigenvectors of L_n for h = 1.

    Returns ``(lam, V)`` with ``V[:, k]`` the eigenvector of ``lam[k]``, rows
    indexed by j = 1..n as in the lemmas.  For periodic BC with odd n the
    alternating vector and the eigenvalue 4 are absent (reading of the
    Lemma spectrumP garble: the pairs k = 1..l-1 already give n vectors).
    """
    j = np.arange(1, n + 1, dtype=np.float64)
    lam, cols = [], []
    if bc == "P":
        ell = (n + 1) // 2 if n % 2 else n // 2  # n = 2l-1 or n = 2l
        lam.append(0.0)
        cols.append(np.ones(n))
        for k in range(1, ell):
            x = 2.0 * k * math.pi / n
            lam += [2.0 - 2.0 * math.cos(x)] * 2
            cols.append(np.cos(j * x))
            cols.append(np.sin(j * x))
        if n % 2 == 0:
            lam.append(4.0)
            cols.append(np.where(np.arange(n) % 2 == 0, 1.0, -1.0))
    elif bc == "D":
        for k in range(1, n + 1):
            x = k * math.pi / (n + 1)
            lam.append(2.0 - 2.0 * math.cos(x))
            cols.append(np.sin(j * x))
    elif bc == "N":
        for k in range(1, n + 1):
            x = (k - 1) * math.pi / n
            lam.append(2.0 - 2.0 * math.cos(x))
            cols.append(np.cos((j - 0.5) * x))
    elif bc in ("DN", "ND"):
        for k in range(1, n + 1):
            th = (2 * k - 1) * math.pi / (2 * n + 1)
            lam.append(2.0 - 2.0 * math.cos(th))
            if bc == "DN":
                cols.append(np.sin(j * th - k * math.pi))
            else:
                cols.append(np.cos(j * th - th / 2.0))
    else:
        raise ValueError(f"unknown boundary condition {bc!r}")
    return np.asarray(lam), np.stack(cols, axis=1)


# --------------------------------------------------------------------------
# Sec. 3.3: 2D/3D operator
# --------------------------------------------------------------------------
def axis_matrices(shape, bcs, hs):
    """The three 1D operators L_n, L_q, L_t (absent axis -> 1x1 zero)."""
    out = []
    for ell, bc, h in zip(shape, bcs, hs):
        out.append(lap1d(ell, None if ell == 1 else bc, h))
    return out


def kron_sum(shape, bcs, hs=(1.0, 1.0, 1.0)) -> sp.csr_matrix:
    """Assembled L_3D = I_t(x)I_q(x)L_n + I_t(x)L_q(x)I_n + L_t(x)I_q(x)I_n (eq. ourproblem2)."""
    n, q, t = shape
    Ln, Lq, Lt = (sp.csr_matrix(M) for M in axis_matrices(shape, bcs, hs))
    In, Iq, It = sp.identity(n), sp.identity(q), sp.identity(t)
    L = sp.kron(It, sp.kron(Iq, Ln)) + sp.kron(It, sp.kron(Lq, In)) + sp.kron(Lt, sp.kron(Iq, In))
    return sp.csr_matrix(L)


def mode_product(M: np.ndarray, U: np.ndarray, mode: int) -> np.ndarray:
    """M x_mode U: multiply every mode-``mode`` fibre of U by M (Sec. 2.2)."""
    moved = np.moveaxis(U, mode, 0)
    out = np.tensordot(M, moved, axes=(1, 0))
    return np.moveaxis(out, 0, mode)


def apply_minus_laplacian(U: np.ndarray, Ls) -> np.ndarray:
    """-Delta_FD(U) = L_n x_1 U + L_q x_2 U + L_t x_3 U (eq. ourproblem), dense mode products."""
    return sum(mode_product(Ls[m], U, m) for m in range(3))


def vec(U: np.ndarray) -> np.ndarray:
    """vec(U): first index fastest (Sec. 2.1)."""
    return U.ravel(order="F")


def unvec(x: np.ndarray, shape) -> np.ndarray:
    return x.reshape(shape, order="F")


def is_singular(shape, bcs) -> bool:
    """L_3D is singular iff every present axis is P or N (end of Sec. 3.3)."""
    return all(ell == 1 or bc in ("P", "N") for ell, bc in zip(shape, bcs))


# --------------------------------------------------------------------------
# Sec. 3.4: right-hand side
# --------------------------------------------------------------------------
def center(X: np.ndarray) -> np.ndarray:
    """Project out the constant (null-space) direction: X - mean(X) (eq. centering)."""
    return X - X.sum() / X.size


def rhs_add_bc(H: np.ndarray, bcs, hs, bvals) -> np.ndarray:
    """Fold nonhomogeneous D/N boundary data into the right-hand side (Sec. 3.4.2).

    ``bvals[2*m]`` is the value at the start face of axis m, ``bvals[2*m+1]``
    at the end face.  A Dirichlet face adds u_B / h^2 to the first (or last)
    layer; a Neumann face adds e_B / h (e_B read as the outward normal
    derivative).  Periodic faces take no data.
    """
    H = H.copy()
    for m in range(3):
        ell = H.shape[m]
        if ell == 1:
            continue
        bc, h = bcs[m], hs[m]
        if bc == "P":
            continue
        start_kind, end_kind = {"D": ("D", "D"), "N": ("N", "N"), "DN": ("D", "N"), "ND": ("N", "D")}[bc]
        for face, kind, idx in ((0, start_kind, 0), (1, end_kind, ell - 1)):
            v = bvals[2 * m + face]
            add = v / (h * h) if kind == "D" else v / h
            sl = [slice(None)] * 3
            sl[m] = idx
            H[tuple(sl)] += add
    return H


_FACE_KINDS = {"D": ("D", "D"), "N": ("N", "N"), "DN": ("D", "N"), "ND": ("N", "D")}


def efield(U: np.ndarray, bcs, hs, bvals=None):
    """epsilon = -grad(ups) (Sec. 2), one array per present axis.

    Second-order central differences  -(u_{i+1} - u_{i-1}) / (2 h).  The neighbour
    across a face is the ghost value that eq. (lap1d) and Sec. 3.4.2 imply:
    periodic faces wrap; a Dirichlet face holds u_B; a Neumann face holds
    u_boundary + h * e_B with e_B the outward normal derivative (so e_B = 0 is the
    mirror value of the homogeneous problem).  ``bvals`` as in ``rhs_add_bc``
    (None: homogeneous data).
    """
    U = np.asarray(U, dtype=np.float64)
    out = []
    for m in range(3):
        ell = U.shape[m]
        if ell == 1:
            continue
        bc, h = bcs[m], hs[m]
        u = np.moveaxis(U, m, 0)
        if bc == "P":
            lo, hi = u[-1:], u[:1]
        else:
            sk, ek = _FACE_KINDS[bc]
            vs = 0.0 if bvals is None else bvals[2 * m]
            ve = 0.0 if bvals is None else bvals[2 * m + 1]
            lo = np.full_like(u[:1], vs) if sk == "D" else u[:1] + h * vs
            hi = np.full_like(u[-1:], ve) if ek == "D" else u[-1:] + h * ve
        ext = np.concatenate([lo, u, hi], axis=0)
        out.append(np.moveaxis(-(ext[2:] - ext[:-2]) / (2.0 * h), 0, m))
    return out


def normalize_rhs(H: np.ndarray) -> np.ndarray:
    """Scale so that ||vec(H)||_2 = 1 / (number of grid points) (eq. normalization)."""
    return H * ((1.0 / H.size) / np.linalg.norm(H.ravel()))


# --------------------------------------------------------------------------
# Sec. 4.3.3, Algorithms 4-7: Moore-Penrose pseudoinverse preconditioner
# --------------------------------------------------------------------------
def pinv_init(shape, bcs, hs=(1.0, 1.0, 1.0), threshold: float | None = None):
    """Algorithm 5 (Algorithm 4 for t = 1): eig of each L_l, then the Hadamard
    pseudoinverse G of all eigenvalue sums, sums below the threshold set to 0.

    Returns ``(Vs, lams, G)``; V_l has orthonormal columns (eq. eig-svd-decomp).
    """
    Ls = axis_matrices(shape, bcs, hs)
    Vs, lams = [], []
    for L in Ls:
        lam, V = np.linalg.eigh(L)
        Vs.append(V)
        lams.append(lam)
    if threshold is None:
        threshold = PINV_THRESHOLD * max(1.0 / (h * h) for h in hs)
    S = lams[0][:, None, None] + lams[1][None, :, None] + lams[2][None, None, :]
    G = np.zeros_like(S)
    keep = np.abs(S) >= threshold
    G[keep] = 1.0 / S[keep]
    return Vs, lams, G


def pinv_apply(R: np.ndarray, Vs, G: np.ndarray) -> np.ndarray:
    """Algorithm 7: F1 = (Vn^T, Vq^T, Vt^T | R); F2 = F1 (.) G; Z = (Vn, Vq, Vt | F2)."""
    F1 = R
    for m in range(3):
        F1 = mode_product(Vs[m].T, F1, m)
    F2 = F1 * G
    F3 = F2
    for m in range(3):
        F3 = mode_product(Vs[m], F3, m)
    return F3


# --------------------------------------------------------------------------
# Sec. 4.1, Algorithm 1: PCG
# --------------------------------------------------------------------------
class PCGResult:
    def __init__(self, U, iters, true_res, recur_res, alphas, removed_mean, null_component):
        self.U = U
        self.iters = iters
        self.true_res = true_res          # relative true residual per iterate (s = 0..iters)
        self.recur_res = recur_res        # relative recurrence residual ||R_s|| / ||H||
        self.alphas = alphas
        self.removed_mean = removed_mean
        self.null_component = null_component


def jacobi_init(shape, bcs, hs, omega):
    """Precomputed parts of the Jacobi(p, omega) preconditioner (Sec. 4.3.1): the
    splitting L_l = D_omega(L_l) + O_omega(L_l) with D_omega = omega * diag(L_l) and
    O_omega = L_l - D_omega per axis, and the Hadamard inverse of the tensor of
    summed diagonals times omega (eq. HadInv and its 3D analogue)."""
    Ls = axis_matrices(shape, bcs, hs)
    Os = [L - omega * np.diag(np.diag(L)) for L in Ls]
    d = [np.diag(L) for L in Ls]
    Dhat = omega * (d[0][:, None, None] + d[1][None, :, None] + d[2][None, None, :])
    return Os, 1.0 / Dhat


def jacobi_apply(R: np.ndarray, Os, Dinv: np.ndarray, p: int) -> np.ndarray:
    """Algorithm 3: X_0 = 0; X_j = Dinv (Hadamard) (R - sum_l O_omega(L_l) x_l X_{j-1}); Z = X_p."""
    X = np.zeros_like(R)
    for _ in range(p):
        F = R - sum(mode_product(Os[m], X, m) for m in range(3))
        X = Dinv * F
    return X


def pcg(shape, bcs, hs, H, U0=None, tol=1e-13, maxit=50, precond="pinv", L=None, pinv=None, jacobi=(3, 1.3),
        patience=None):
    """Algorithm 1 with the pseudoinverse preconditioner (Algorithm 7).

    The Laplacian is the assembled sparse Kronecker sum (not a stencil).  If
    the operator is singular, H is centred once (eq. centering) and Z_s every
    iteration (Remark orthogonality); U is centred at exit so that the
    zero-mean (minimum-norm) representative is returned.  ``precond`` is
    ``"pinv"``, ``"jacobi"`` (Algorithm 3 with ``jacobi = (p, omega)``) or
    ``"none"`` (M = I).  Stops when the true relative residual is <= tol, at
    maxit, or on stagnation: ``patience`` consecutive iterations without halving
    the best true residual (default 3 for the pseudoinverse, whose residual
    falls by orders of magnitude per step; 50 for the comparators, whose CG
    residual is not monotone).
    """
    if patience is None:
        patience = 3 if precond == "pinv" else 50
    if L is None:
        L = kron_sum(shape, bcs, hs)
    singular = is_singular(shape, bcs)
    if precond == "pinv":
        Vs, _, G = pinv if pinv is not None else pinv_init(shape, bcs, hs)

        def M(R):
            Z = pinv_apply(R, Vs, G)
            return center(Z) if singular else Z
    elif precond == "jacobi":
        jp, omega = jacobi
        Os, Dinv = jacobi_init(shape, bcs, hs, omega)

        def M(R):
            Z = jacobi_apply(R, Os, Dinv, jp)
            return center(Z) if singular else Z
    else:

        def M(R):
            return center(R) if singular else R.copy()

    def apply_L(X):
        return unvec(L @ vec(X), shape)

    H = np.asarray(H, dtype=np.float64)
    removed_mean = 0.0
    if singular:
        removed_mean = H.sum() / H.size
        H = center(H)
    hnorm = np.linalg.norm(H.ravel())
    if hnorm == 0.0:
        return PCGResult(np.zeros(shape), 0, [0.0], [0.0], [], removed_mean, 0.0)
    U = np.zeros(shape) if U0 is None else np.array(U0, dtype=np.float64)
    W = apply_L(U)                                  # L U_0
    R = H - W                                       # initial residual
    Z = M(R)                                        # preconditioned residual
    rho = float(np.vdot(R, Z))                      # rho_0 = <R_0, Z_0>
    P = Z.copy()                                    # first direction
    true_res = [np.linalg.norm((H - apply_L(U)).ravel()) / hnorm]
    recur_res = [np.linalg.norm(R.ravel()) / hnorm]
    alphas = []
    s = 0
    best = true_res[0]
    stall = 0
    while true_res[-1] > tol and s < maxit:
        s += 1                                      # iteration counter
        W = apply_L(P)                              # W = L P
        alpha = rho / float(np.vdot(W, P))          # step length
        U = U + alpha * P                           # iterate update
        R = R - alpha * W                           # residual recurrence
        Z = M(R)                                    # preconditioner
        rho_new = float(np.vdot(R, Z))              # new rho
        beta = rho_new / rho                        # beta (ratio of rhos)
        P = Z + beta * P                            # next direction
        rho = rho_new
        alphas.append(alpha)
        true_res.append(np.linalg.norm((H - apply_L(U)).ravel()) / hnorm)
        recur_res.append(np.linalg.norm(R.ravel()) / hnorm)
        if true_res[-1] < 0.5 * best:
            best, stall = true_res[-1], 0
        else:
            stall += 1
            if stall >= patience:
                break
    null_component = 0.0
    if singular:
        null_component = U.sum() / U.size
        U = center(U)
    return PCGResult(U, s, true_res, recur_res, alphas, removed_mean, null_component)


# --------------------------------------------------------------------------
# Direct cross-checks of the same definition (minimum-norm solution L^+ H)
# --------------------------------------------------------------------------
def minnorm_dense(shape, bcs, hs, H, threshold=1e-10):
    """Brute force for tiny grids: dense symmetric eigendecomposition of the
    assembled operator, eigenvalues below ``threshold * max|eig|`` treated as 0.
    Returns the minimum-norm solution L^+ vec(H) (Sec. 4.3.2, eq. p-inv-full)."""
    L = kron_sum(shape, bcs, hs).toarray()
    w, Q = np.linalg.eigh(L)
    cut = threshold * np.max(np.abs(w))
    winv = np.where(np.abs(w) > cut, 1.0 / np.where(np.abs(w) > cut, w, 1.0), 0.0)
    x = Q @ (winv * (Q.T @ vec(H)))
    return unvec(x, shape)


def solve_sparse_direct(shape, bcs, hs, H):
    """Nonsingular operators only: scipy sparse LU solve of L vec(U) = vec(H)."""
    import scipy.sparse.linalg as spla

    L = kron_sum(shape, bcs, hs).tocsc()
    return unvec(spla.spsolve(L, vec(H)), shape)


# --------------------------------------------------------------------------
# Cost model of Tables PCGcost and PInvPcost (operation counts)
# --------------------------------------------------------------------------
def pinv_apply_flops(n, q, t):
    """Table PInvPcost: one application costs 4nqt(n+q+t+1/4) operations (3D)."""
    return 4 * n * q * t * (n + q + t + 0.25)


def pcg_iteration_flops_sparse(n, q, t):
    """Table PCGcost, sparse Laplacian: 28nqt per iteration (3D), preconditioner excluded."""
    return 28 * n * q * t
