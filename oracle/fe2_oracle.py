"""FP64 CPU oracle for the per-Gauss-point RVE block of monolithic FE^2.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no
code with the CUDA path and never imports the product package.

What it computes (Hesch, Schmidt & Schuss, arXiv 2312.12771):

* Section 2.1, cofactor and determinant equations: H = 1/2 F x F (tensor cross
  product with Levi-Civita symbols), J = 1/6 F : (F x F).
* Section 2.1, Eq. (MR) and the P formula below it: the compressible
  Mooney-Rivlin law with the f(J) of the Section 5.2 membrane materials
  (mooney_rivlin), and with beta = 0 the compressible Neo-Hooke law,
  Psi = mu/2 (F:F - 3) - mu ln J + kappa/2 (J-1)^2 (3D; plane strain embeds
  F with F33 = 1), P = dPsi/dF, A = dP/dF.
* Section 2.2, Eqs. (microdefo), (microGrad): F~ = Fbar + grad w~.
* Section 2.2, Eq. (Con)(iii): periodic fluctuations; the corner node is
  pinned (Section 5.2 fixes the four corners, which periodicity identifies).
* Section 3, Eqs. (linSys3), (linSys4): micro residual and the volume-averaged
  stress with full 2^d Gauss quadrature of bilinear / trilinear elements.
* Section 4, Eqs. (discreteSys_K), (discreteSys_D), (discreteSys_L): the
  Hessian blocks, here per RVE: K_MM = int A, K_mM = int grad(R)^T A,
  K_mm = int grad(R)^T A grad(R).
* Section 3, Eqs. (constSolution1), (constSolution2): the piecewise-constant
  macro basis for w~, one RVE per macro element (rve_solve_elem).
* Section 4.1: the classical staggered (nested) FE^2 scheme, with an inner
  micro Newton to equilibrium in every macro iteration (staggered_fe2).
* Section 4.2, Eq. (solution2) and the update of w~ below it: the condensed
  (null-space reduced) tangent Cbar = (K_MM - K_Mm K_mm^-1 K_mM)/|Omega|, the
  effective stress sigma_eff = (Pint - K_Mm K_mm^-1 r_m)/|Omega| and
  dw~ = -(x_r + X_M : dFbar).

Everything is plain FP64 numpy; the Cholesky factorisation and triangular
solves are LAPACK calls through scipy (library primitives).  DOFs use the
natural periodic numbering p = i + N j (+ N^2 k), reduced DOF d*(p-1)+c.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.linalg
import scipy.sparse

# ---------------------------------------------------------------------------
# Section 2.1: tensor cross product, cofactor, determinant
# ---------------------------------------------------------------------------
_EPS = np.zeros((3, 3, 3))
for _i, _j, _k in itertools.permutations(range(3)):
    _EPS[_i, _j, _k] = np.linalg.det(np.eye(3)[[_i, _j, _k]])


def tensor_cross(A, B):
    """[A x B]_iJ = eps_ijk eps_JMN A_jM B_kN  (Section 2.1)."""
    return np.einsum("ijk,JMN,...jM,...kN->...iJ", _EPS, _EPS, A, B)


def cofactor(F):
    """H = 1/2 F x F  (Section 2.1, cofactor equation)."""
    return 0.5 * tensor_cross(F, F)


def jacobian(F):
    """J = 1/6 F : (F x F)  (Section 2.1, determinant equation)."""
    return np.einsum("...iJ,...iJ->...", F, tensor_cross(F, F)) / 6.0


def embed3(F, d):
    """Plane strain: a 2x2 gradient is embedded with F33 = 1."""
    if d == 3:
        return F
    F3 = np.zeros(F.shape[:-2] + (3, 3), dtype=F.dtype)
    F3[..., :2, :2] = F
    F3[..., 2, 2] = 1.0
    return F3


# ---------------------------------------------------------------------------
# constitutive laws (3D, restricted to the in-plane block for d = 2)
# ---------------------------------------------------------------------------
def neohooke_energy(F, mu, kappa, d):
    """Psi = mu/2 (F:F - 3) - mu ln J + kappa/2 (J-1)^2 -- Eq. (MR) with
    alpha = mu/2, beta = 0 and f(J) = -mu ln J + kappa/2 (J-1)^2."""
    F3 = embed3(F, d)
    J = jacobian(F3)
    return 0.5 * mu * (np.einsum("...iJ,...iJ->...", F3, F3) - 3.0) - mu * np.log(J) \
        + 0.5 * kappa * (J - 1.0) ** 2


def neohooke(F, mu, kappa, d):
    """P = dPsi/dF + dPsi/dJ H (Section 2.1, P formula with beta = 0) and
    A = dP/dF = mu I + (mu/J^2 + kappa) H (x) H + (kappa (J-1) - mu/J) dH/dF,
    with dH/dF : dF = F x dF."""
    F3 = embed3(F, d)
    H = cofactor(F3)
    J = jacobian(F3)
    s = kappa * (J - 1.0) - mu / J                      # dPsi/dJ
    P = mu * F3 + s[..., None, None] * H
    I4 = np.einsum("ik,JL->iJkL", np.eye(3), np.eye(3))
    dHdF = np.einsum("ijk,JML,...jM->...iJkL", _EPS, _EPS, F3)
    A = mu * I4 + (mu / J ** 2 + kappa)[..., None, None, None, None] * \
        np.einsum("...iJ,...kL->...iJkL", H, H) + s[..., None, None, None, None] * dHdF
    return P[..., :d, :d], A[..., :d, :d, :d, :d]


def mooney_rivlin_energy(F, alpha, beta, kappa, d):
    """Psi = alpha (F:F - 3) + beta (H:H - 3) + kappa/2 (J-1)^2 - 2 (alpha + 2 beta) ln J:
    Eq. (MR) with the f(J) of the Section 5.2 membrane materials (stress free
    at F = I).  For d = 2 the plane-strain embedding gives H:H = F:F + J^2,
    which is the two-dimensional energy printed in Section 5.2."""
    F3 = embed3(F, d)
    H = cofactor(F3)
    J = jacobian(F3)
    return alpha * (np.einsum("...iJ,...iJ->...", F3, F3) - 3.0) + beta * (np.einsum("...iJ,...iJ->...", H, H) - 3.0) \
        + 0.5 * kappa * (J - 1.0) ** 2 - 2.0 * (alpha + 2.0 * beta) * np.log(J)


def mooney_rivlin(F, alpha, beta, kappa, d):
    """P = dPsi/dF + dPsi/dH x F + dPsi/dJ H (Section 2.1, P formula) with
    dPsi/dF = 2 alpha F, dPsi/dH = 2 beta H, dPsi/dJ = kappa (J-1) - 2 (alpha + 2 beta)/J.
    A = dP/dF from dH : dF = F x dF:
      A:dF = 2 alpha dF + 2 beta ((F x dF) x F + H x dF) + f''(J) (H:dF) H + f'(J) F x dF."""
    F3 = embed3(F, d)
    H = cofactor(F3)
    J = jacobian(F3)
    s = kappa * (J - 1.0) - 2.0 * (alpha + 2.0 * beta) / J          # f'(J)
    c = kappa + 2.0 * (alpha + 2.0 * beta) / J ** 2                 # f''(J)
    P = 2.0 * alpha * F3 + 2.0 * beta * tensor_cross(H, F3) + s[..., None, None] * H
    I4 = np.einsum("ik,JL->iJkL", np.eye(3), np.eye(3))
    dHdF = np.einsum("ijk,JML,...jM->...iJkL", _EPS, _EPS, F3)        # (F x dF)_iJ = dHdF_iJkL dF_kL
    HxdF = np.einsum("ijk,JML,...jM->...iJkL", _EPS, _EPS, H)        # (H x dF)_iJ
    # ((F x dF) x F)_iJ = eps_ijk eps_JMN (F x dF)_jM F_kN
    FdFxF = np.einsum("ijk,JMN,...jMbD,...kN->...iJbD", _EPS, _EPS, dHdF, F3)
    A = 2.0 * alpha * I4 + 2.0 * beta * (FdFxF + HxdF) \
        + c[..., None, None, None, None] * np.einsum("...iJ,...kL->...iJkL", H, H) \
        + s[..., None, None, None, None] * dHdF
    return P[..., :d, :d], A[..., :d, :d, :d, :d]


def lame(E, nu):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def linear_energy(F, E, nu, d):
    """Psi = 1/2 eps : C : eps, eps = sym(F - I), isotropic C (plane strain for d=2)."""
    lam, mu = lame(E, nu)
    eps = 0.5 * (F + np.swapaxes(F, -1, -2)) - np.eye(d)
    tr = np.einsum("...ii->...", eps)
    return 0.5 * lam * tr ** 2 + mu * np.einsum("...ij,...ij->...", eps, eps)


def linear_elastic(F, E, nu, d):
    """sigma = lam tr(eps) I + 2 mu eps, A_iJkL = lam d_iJ d_kL + mu (d_ik d_JL + d_iL d_Jk)."""
    lam, mu = lame(E, nu)
    eps = 0.5 * (F + np.swapaxes(F, -1, -2)) - np.eye(d)
    tr = np.einsum("...ii->...", eps)
    P = lam * tr[..., None, None] * np.eye(d) + 2.0 * mu * eps
    I = np.eye(d)
    A = lam * np.einsum("iJ,kL->iJkL", I, I) + mu * (np.einsum("ik,JL->iJkL", I, I)
                                                     + np.einsum("iL,Jk->iJkL", I, I))
    A = np.broadcast_to(A, F.shape[:-2] + (d, d, d, d)).copy()
    return P, A


def material(F, m, d):
    """Dispatch on the material row m = (model, p1, p2, p3)."""
    model = int(m[0])
    if model == 0:
        return linear_elastic(F, m[1], m[2], d)
    if model == 1:
        return neohooke(F, m[1], m[2], d)
    if model == 2:
        return mooney_rivlin(F, m[1], m[2], m[3], d)
    raise ValueError(f"unknown material model {model}")


def energy(F, m, d):
    model = int(m[0])
    if model == 0:
        return linear_energy(F, m[1], m[2], d)
    if model == 2:
        return mooney_rivlin_energy(F, m[1], m[2], m[3], d)
    return neohooke_energy(F, m[1], m[2], d)


# ---------------------------------------------------------------------------
# Section 3: bilinear / trilinear elements with 2^d Gauss points
# ---------------------------------------------------------------------------
def local_nodes(d):
    """Local node a <-> offset bits (a_x, a_y[, a_z]) with a = a_x + 2 a_y + 4 a_z."""
    return np.array([[(a >> k) & 1 for k in range(d)] for a in range(2 ** d)])


def gauss_grads(d, h):
    """Shape-function gradients dN_a/dX_J at the 2^d Gauss points of a cube
    element of side h, and the quadrature weight (h/2)^d of each point."""
    g = 1.0 / math.sqrt(3.0)
    offs = local_nodes(d)
    s = 2.0 * offs - 1.0                              # node signs in [-1,1]^d
    G = np.zeros((2 ** d, 2 ** d, d))
    for q, bits in enumerate(local_nodes(d)):
        xi = g * (2.0 * bits - 1.0)
        for a in range(2 ** d):
            for J in range(d):
                val = 0.5 * s[a, J]
                for K in range(d):
                    if K != J:
                        val *= 0.5 * (1.0 + s[a, K] * xi[K])
                G[q, a, J] = val * 2.0 / h
    return G, (h / 2.0) ** d


def full_grid(N, d):
    """Full (non-periodic) nodal grid (N+1)^d with element connectivity."""
    n1 = N + 1
    strides = [n1 ** k for k in range(d)]
    offs = local_nodes(d)
    elems = []
    for e in range(N ** d):
        ec = [(e // N ** k) % N for k in range(d)]
        elems.append([sum((ec[k] + offs[a, k]) * strides[k] for k in range(d))
                      for a in range(2 ** d)])
    return np.array(elems, dtype=np.int64), n1 ** d


def periodic_T(N, d):
    """Discrete null-space matrix of periodicity with the corner pinned
    (Section 2.2, Eq. (Con)(iii); Section 5.2): a 0/1 matrix mapping the
    reduced DOFs to the full-grid DOFs."""
    n1 = N + 1
    nfull = n1 ** d
    rows, cols = [], []
    for node in range(nfull):
        ijk = [(node // n1 ** k) % n1 for k in range(d)]
        p = sum((ijk[k] % N) * N ** k for k in range(d))
        if p == 0:
            continue                                     # pinned corner
        for c in range(d):
            rows.append(d * node + c)
            cols.append(d * (p - 1) + c)
    nm = d * (N ** d - 1)
    return scipy.sparse.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(d * nfull, nm))


# ---------------------------------------------------------------------------
# Section 3 / 4: RVE integrals, periodic reduction, condensation
# ---------------------------------------------------------------------------
def rve_integrals(N, d, phase, mat, Fbar, w=None, L=1.0):
    """Assemble the unreduced RVE quantities on the full grid at (Fbar, w~):
    K (Hessian wrt w~), f (micro residual), KM (d f / d Fbar), K_MM = int A,
    Pint = int P~  (Eqs. (linSys3), (linSys4), (discreteSys_K/D/L))."""
    h = L / N
    G, wq = gauss_grads(d, h)
    conn, nnode = full_grid(N, d)
    T = periodic_T(N, d)
    nm = T.shape[1]
    w = np.zeros(nm) if w is None else np.asarray(w, dtype=np.float64)
    wfull = (T @ w).reshape(nnode, d)
    we = wfull[conn]                                    # [ne][2^d][d]
    ne, na = conn.shape
    # F~ at every (element, gauss point): Fbar + sum_a w_a (x) grad N_a
    Ft = Fbar[None, None] + np.einsum("eai,qaJ->eqiJ", we, G)
    P = np.zeros_like(Ft)
    A = np.zeros(Ft.shape[:2] + (d, d, d, d))
    for ph in np.unique(phase):
        sel = phase == ph
        P[sel], A[sel] = material(Ft[sel], mat[ph], d)
    ke = np.einsum("qaJ,eqiJkL,qbL->eaibk", G, A, G) * wq
    fe = np.einsum("eqiJ,qaJ->eai", P, G) * wq
    kMe = np.einsum("qaJ,eqiJkL->eaikL", G, A) * wq
    K_MM = A.sum(axis=(0, 1)).reshape(d * d, d * d) * wq
    Pint = P.sum(axis=(0, 1)).reshape(d * d) * wq
    nd = d * nnode
    dof = (d * conn[:, :, None] + np.arange(d)[None, None, :]).reshape(ne, na * d)
    rr = np.repeat(dof[:, :, None], na * d, axis=2)
    cc = np.repeat(dof[:, None, :], na * d, axis=1)
    K = scipy.sparse.coo_matrix((ke.reshape(ne, -1).ravel(), (rr.ravel(), cc.ravel())),
                                shape=(nd, nd)).tocsr()
    f = np.zeros(nd)
    np.add.at(f, dof.ravel(), fe.reshape(-1))
    KM = np.zeros((nd, d * d))
    np.add.at(KM, dof.ravel(), kMe.reshape(ne * na * d, d * d))
    return dict(K=K, f=f, KM=KM, K_MM=K_MM, Pint=Pint, T=T, vol=L ** d, Ft=Ft, P=P, G=G, wq=wq)


def reduce_periodic(ints):
    """K_mm = T^T K T, r_m = T^T f, K_mM = T^T KM  (null space of periodicity)."""
    T = ints["T"]
    K_mm = (T.T @ ints["K"] @ T).toarray()
    r_m = T.T @ ints["f"]
    K_mM = T.T @ ints["KM"]
    return K_mm, r_m, K_mM


def condense(K_mm, r_m, K_mM, K_MM, Pint, vol):
    """Section 4.2, Eq. (solution2): Cbar = (K_MM - K_Mm K_mm^-1 K_mM)/|Omega|,
    sigma_eff = (Pint - K_Mm K_mm^-1 r_m)/|Omega|, with X_M = K_mm^-1 K_mM and
    x_r = K_mm^-1 r_m (dense Cholesky)."""
    cf = scipy.linalg.cho_factor(K_mm, lower=True)
    X = scipy.linalg.cho_solve(cf, np.column_stack([K_mM, r_m]))
    X_M, x_r = X[:, :-1], X[:, -1]
    Cbar = (K_MM - K_mM.T @ X_M) / vol
    sigma = (Pint - K_mM.T @ x_r) / vol
    return dict(Cbar=Cbar, sigma_eff=sigma, X_M=X_M, x_r=x_r, Pbar=Pint / vol)


def rve_solve(N, d, phase, mat, Fbar, w=None, L=1.0):
    """One RVE solve (S1-S6): integrals -> periodic reduction -> condensation."""
    ints = rve_integrals(N, d, np.asarray(phase), np.asarray(mat), np.asarray(Fbar, float), w, L)
    K_mm, r_m, K_mM = reduce_periodic(ints)
    out = condense(K_mm, r_m, K_mM, ints["K_MM"], ints["Pint"], ints["vol"])
    out.update(K_mm=K_mm, r_m=r_m, K_mM=K_mM, K_MM=ints["K_MM"], Pint=ints["Pint"])
    return out


def rve_solve_elem(N, d, phase, mat, Fbars, wq, w=None, L=1.0):
    """Piecewise-constant macro basis for w~ (Section 3, Eqs. (constSolution1),
    (constSolution2)): one fluctuation w~ per macro element, whose micro
    residual and stiffness are integrated over the element's macro Gauss
    points q (deformation gradients Fbars[q], weights wq normalised to sum 1):
      K_mm = sum_q wq K_mm(Fbar_q),  r_m = sum_q wq r_m(Fbar_q),  K_mM,q = K_mM(Fbar_q).
    Condensing dw~ = -K_mm^-1 (r_m + sum_q wq K_mM,q : dFbar_q) gives per pair
    of Gauss points (q, q') the d^2 x d^2 block
      Cbar[q][q'] = (K_MM,q delta_qq' - K_Mm,q K_mm^-1 K_mM,q' wq')/|Omega|
    and sigma_eff,q = (Pint_q - K_Mm,q K_mm^-1 r_m)/|Omega|.  With one Gauss
    point this is rve_solve."""
    nq = len(Fbars)
    wq = np.asarray(wq, dtype=np.float64)
    parts = []
    for q in range(nq):
        ints = rve_integrals(N, d, np.asarray(phase), np.asarray(mat), np.asarray(Fbars[q], float), w, L)
        K_q, r_q, KmM_q = reduce_periodic(ints)
        parts.append((K_q, r_q, KmM_q, ints["K_MM"], ints["Pint"], ints["vol"]))
    K_mm = sum(wq[q] * parts[q][0] for q in range(nq))
    r_m = sum(wq[q] * parts[q][1] for q in range(nq))
    vol = parts[0][5]
    cf = scipy.linalg.cho_factor(K_mm, lower=True)
    X = [scipy.linalg.cho_solve(cf, parts[q][2]) for q in range(nq)]
    x_r = scipy.linalg.cho_solve(cf, r_m)
    dd = d * d
    Cbar = np.zeros((nq * dd, nq * dd))
    for q in range(nq):
        for q2 in range(nq):
            blk = -wq[q2] * parts[q][2].T @ X[q2]
            if q == q2:
                blk = blk + parts[q][3]
            Cbar[q * dd:(q + 1) * dd, q2 * dd:(q2 + 1) * dd] = blk / vol
    sigma = np.array([(parts[q][4] - parts[q][2].T @ x_r) / vol for q in range(nq)])
    return dict(Cbar=Cbar, sigma_eff=sigma, X_M=X, x_r=x_r, r_m=r_m, K_mm=K_mm,
                Pbar=np.array([parts[q][4] / vol for q in range(nq)]))


def micro_equilibrate_elem(N, d, phase, mat, Fbars, wq, w=None, tol=1e-13, maxit=50, L=1.0):
    """Inner Newton on one element RVE (piecewise-constant basis) at fixed
    Fbars until ||r_m|| < tol, r_m = sum_q wq r_m(Fbar_q)."""
    nm = d * (N ** d - 1)
    w = np.zeros(nm) if w is None else np.array(w, dtype=np.float64)
    for it in range(maxit):
        s = rve_solve_elem(N, d, phase, mat, Fbars, wq, w, L)
        if np.linalg.norm(s["r_m"]) < tol:
            return w, it
        w = w - s["x_r"]
    raise RuntimeError("micro Newton did not converge")


def micro_equilibrate(N, d, phase, mat, Fbar, w=None, tol=1e-13, maxit=50, L=1.0, history=None):
    """Classical inner Newton on one RVE at fixed Fbar (Section 4.1) until
    ||r_m|| < tol; returns the equilibrium fluctuation and iteration count.
    ``history`` (a list, optional) receives its list of ||r_m|| values."""
    nm = d * (N ** d - 1)
    w = np.zeros(nm) if w is None else np.array(w, dtype=np.float64)
    mine = []
    if history is not None:
        history.append(mine)
    for it in range(maxit):
        ints = rve_integrals(N, d, phase, mat, Fbar, w, L)
        K_mm, r_m, _ = reduce_periodic(ints)
        mine.append(float(np.linalg.norm(r_m)))
        if np.linalg.norm(r_m) < tol:
            return w, it
        w = w - scipy.linalg.cho_solve(scipy.linalg.cho_factor(K_mm, lower=True), r_m)
    raise RuntimeError("micro Newton did not converge")


# ---------------------------------------------------------------------------
# Section 3 / 4.2: macro Q4 problem and the monolithic (generalised) Newton
# ---------------------------------------------------------------------------
def macro_mesh(nx, ny, Lx=1.0, Ly=1.0):
    xs = np.linspace(0.0, Lx, nx + 1)
    ys = np.linspace(0.0, Ly, ny + 1)
    X = np.array([[x, y] for y in ys for x in xs])
    conn = []
    for ey in range(ny):
        for ex in range(nx):
            n0 = ex + (nx + 1) * ey
            conn.append([n0, n0 + 1, n0 + nx + 1, n0 + nx + 2])   # a = ax + 2 ay
    conn = np.array(conn)
    bnd = np.array([i for i, (x, y) in enumerate(X)
                    if abs(x) < 1e-12 or abs(y) < 1e-12 or abs(x - Lx) < 1e-12 or abs(y - Ly) < 1e-12])
    return X, conn, bnd


def macro_mesh3(nx, ny, nz, Lx=1.0, Ly=1.0, Lz=1.0):
    """Hex8 macro mesh of the box: nodes x fastest, then y, then z; local node
    a = a_x + 2 a_y + 4 a_z; returns (X, conn, boundary nodes)."""
    xs, ys, zs = np.linspace(0.0, Lx, nx + 1), np.linspace(0.0, Ly, ny + 1), np.linspace(0.0, Lz, nz + 1)
    X = np.array([[x, y, z] for z in zs for y in ys for x in xs])
    offs = local_nodes(3)
    conn = []
    for ez in range(nz):
        for ey in range(ny):
            for ex in range(nx):
                conn.append([(ex + o[0]) + (nx + 1) * ((ey + o[1]) + (ny + 1) * (ez + o[2])) for o in offs])
    conn = np.array(conn)
    L = (Lx, Ly, Lz)
    bnd = np.array([i for i, x in enumerate(X) if any(abs(x[k]) < 1e-12 or abs(x[k] - L[k]) < 1e-12
                                                       for k in range(3))])
    return X, conn, bnd


def macro_gauss(X, conn):
    """Per macro Gauss point b = 2^d e + q (q = q_x + 2 q_y [+ 4 q_z], 2^d Gauss
    points on the isoparametric Q4 / Hex8): grad N^A(X_b) [2^d][d], weight
    eta_b = det(dX/dxi) and the point X_b."""
    X = np.asarray(X, float)
    d = X.shape[1]
    g = 1.0 / math.sqrt(3.0)
    offs = local_nodes(d)
    s = 2.0 * offs - 1.0
    na = 2 ** d
    grads, etas, pts = [], [], []
    for e in range(len(conn)):
        xe = X[conn[e]]
        for bits in offs:
            xi = g * (2.0 * bits - 1.0)
            # N_a = prod_k (1 + s_ak xi_k)/2, dN_a/dxi_J = s_aJ/2 prod_{k != J} (1 + s_ak xi_k)/2
            fac = 0.5 * (1.0 + s * xi[None, :])          # [na][d]
            Nv = np.prod(fac, axis=1)
            dN = np.zeros((na, d))
            for a in range(na):
                for J in range(d):
                    dN[a, J] = 0.5 * s[a, J] * np.prod([fac[a, k] for k in range(d) if k != J])
            Jm = xe.T @ dN                                  # dX/dxi
            grads.append(dN @ np.linalg.inv(Jm))
            etas.append(np.linalg.det(Jm))
            pts.append(Nv @ xe)
    return np.array(grads), np.array(etas), np.array(pts)


def macro_B(grad, d):
    """dFbar_iJ / dq_(A,k) of F_iJ = sum_A q_Ai dN_A/dX_J at one Gauss point:
    row iJ = d i + J, column d A + k."""
    na = grad.shape[0]
    Bm = np.zeros((d * d, d * na))
    for A_ in range(na):
        for i in range(d):
            for J in range(d):
                Bm[d * i + J, d * A_ + i] = grad[A_, J]
    return Bm


def macro_system(conn, grads, etas, stress, Cbar, d):
    """Macro tangent and residual of Section 3, Eq. (linSys2) with the condensed
    RVE tangents of Section 4.2, Eq. (solution2):
    K = sum_b eta_b B_b^T Cbar_b B_b,  R = sum_b eta_b B_b^T s_b (dense, all DOFs)."""
    na = 2 ** d
    nnode = int(np.max(conn)) + 1
    Kg = np.zeros((d * nnode, d * nnode))
    Rg = np.zeros(d * nnode)
    for b in range(len(etas)):
        e = b // na
        Bm = macro_B(grads[b], d)
        dofs = (d * np.asarray(conn[e])[:, None] + np.arange(d)[None, :]).ravel()
        Kg[np.ix_(dofs, dofs)] += etas[b] * Bm.T @ np.asarray(Cbar[b]).reshape(d * d, d * d) @ Bm
        Rg[dofs] += etas[b] * Bm.T @ np.asarray(stress[b]).ravel()
    return Kg, Rg


def traction_load(X, edge_nodes, T):
    """Nodal external forces of a constant surface load T on a boundary polyline
    of bilinear-element edges (the Neumann term of Eq. (weakMech)): every
    segment of length L between consecutive nodes gives T L / 2 to each end."""
    f = np.zeros_like(np.asarray(X, dtype=np.float64))
    T = np.asarray(T, dtype=np.float64)
    for a, b in zip(edge_nodes[:-1], edge_nodes[1:]):
        L = np.linalg.norm(X[b] - X[a])
        f[a] += 0.5 * L * T
        f[b] += 0.5 * L * T
    return f


def monolithic_fe2(macro, rves, F_final, n_steps=1, tol_macro=1e-9, tol_micro=1e-9,
                   maxit=25, record=None, fext=None):
    """Load-stepped monolithic Newton (Section 4.2, Eq. (solution2)) on a Q4
    (d = 2) or Hex8 (d = 3) macro mesh with affine Dirichlet data
    u = (F_k - I) X on the nodes ``bnd``, F_k = I + k/n (F_final - I), and
    with ``fext`` (nodal forces [nnode][d] of a surface load, Eq. (weakMech))
    the load k/n fext in step k.  ``rves`` is a list (one per macro Gauss
    point, b = 2^d e + q) of dicts with N, phase, mat.  Returns per Gauss point
    the converged Fbar, sigma (= Pbar), Cbar and w~, plus iteration counts.  A
    step fails when ||R_macro|| > 1e10 (Section 5.2)."""
    X, conn, bnd = macro
    X = np.asarray(X, float)
    d = X.shape[1]
    na = 2 ** d
    grads, etas, _ = macro_gauss(X, conn)
    nb = len(etas)
    nnode = len(X)
    q = X.copy()
    ws = [np.zeros(d * (r["N"] ** d - 1)) for r in rves]
    free = np.ones(d * nnode, bool)
    for n in bnd:
        free[d * n:d * n + d] = False
    iters = []
    for k in range(1, n_steps + 1):
        Fk = np.eye(d) + (k / n_steps) * (np.asarray(F_final) - np.eye(d))
        q[bnd] = X[bnd] @ Fk.T
        for it in range(maxit):
            sols, rmic = [], 0.0
            for b in range(nb):
                e = b // na
                Fb = q[conn[e]].T @ grads[b]
                r = rves[b]
                s = rve_solve(r["N"], d, r["phase"], r["mat"], Fb, ws[b])
                sols.append((Fb, s))
                rmic = max(rmic, np.linalg.norm(s["r_m"]))
            Cb = [s["Cbar"] for _, s in sols]
            Kg, Rg = macro_system(conn, grads, etas, [s["Pbar"] for _, s in sols], Cb, d)     # R_macro
            _, Rc = macro_system(conn, grads, etas, [s["sigma_eff"] for _, s in sols], Cb, d)  # condensed RHS
            if fext is not None:
                Rg -= (k / n_steps) * np.asarray(fext).ravel()
                Rc -= (k / n_steps) * np.asarray(fext).ravel()
            rnorm = np.linalg.norm(Rg[free])
            if record is not None:
                record.append((k, it, rnorm, rmic))
            if rnorm < tol_macro and rmic < tol_micro:
                iters.append(it)
                break
            if not rnorm < 1e10:
                raise RuntimeError("macro residual above 1e10: Newton diverged")
            dq = np.zeros(d * nnode)
            dq[free] = np.linalg.solve(Kg[np.ix_(free, free)], -Rc[free])
            q = q + dq.reshape(nnode, d)
            for b in range(nb):
                e = b // na
                dF = dq.reshape(nnode, d)[conn[e]].T @ grads[b]
                s = sols[b][1]
                ws[b] = ws[b] - (s["x_r"] + s["X_M"] @ dF.ravel())
        else:
            raise RuntimeError("macro Newton did not converge")
    out = []
    for b in range(nb):
        Fb, s = sols[b]
        out.append(dict(Fbar=Fb, Pbar=s["Pbar"], Cbar=s["Cbar"], sigma_eff=s["sigma_eff"], w=ws[b]))
    return out, iters, q


def monolithic_fe2_const(macro, rves, F_final, n_steps=1, tol_macro=1e-9, tol_micro=1e-9,
                         maxit=25, record=None, fext=None):
    """The monolithic Newton of monolithic_fe2 with the piecewise-constant
    macro basis for w~ (Section 3, Eqs. (constSolution1), (constSolution2)):
    ``rves`` holds one RVE per macro element; its solve (rve_solve_elem) uses
    the Fbar of the element's four Gauss points with weights eta_q / sum eta.
    Macro stiffness sum_q sum_q' eta_q B_q^T Cbar[q][q'] B_q', residual
    sum_q eta_q B_q^T Pbar_q, update dw~ = -(x_r + sum_q w_q X_M,q : dFbar_q)."""
    X, conn, bnd = macro
    grads, etas, _ = macro_gauss(X, conn)
    nel = len(conn)
    nnode = len(X)
    q = X.copy()
    ws = [np.zeros(2 * (r["N"] ** 2 - 1)) for r in rves]
    free = np.ones(2 * nnode, bool)
    for n in bnd:
        free[2 * n:2 * n + 2] = False

    def Bmat(b):
        Bm = np.zeros((4, 8))
        for A_ in range(4):
            for i in range(2):
                for J in range(2):
                    Bm[2 * i + J, 2 * A_ + i] = grads[b][A_, J]
        return Bm

    iters = []
    for k in range(1, n_steps + 1):
        Fk = np.eye(2) + (k / n_steps) * (np.asarray(F_final) - np.eye(2))
        q[bnd] = X[bnd] @ Fk.T
        for it in range(maxit):
            Kg = np.zeros((2 * nnode, 2 * nnode))
            Rg = np.zeros(2 * nnode)
            Rc = np.zeros(2 * nnode)
            sols, rmic = [], 0.0
            for e in range(nel):
                bs = [4 * e + g for g in range(4)]
                Fbs = [q[conn[e]].T @ grads[b] for b in bs]
                wq = etas[bs] / etas[bs].sum()
                r = rves[e]
                s = rve_solve_elem(r["N"], 2, r["phase"], r["mat"], Fbs, wq, ws[e])
                sols.append((Fbs, wq, s))
                rmic = max(rmic, np.linalg.norm(s["r_m"]))
                dofs = np.array([[2 * conn[e][A_], 2 * conn[e][A_] + 1] for A_ in range(4)]).ravel()
                for g in range(4):
                    Bg = Bmat(bs[g])
                    Rg[dofs] += etas[bs[g]] * Bg.T @ s["Pbar"][g].ravel()
                    Rc[dofs] += etas[bs[g]] * Bg.T @ s["sigma_eff"][g].ravel()
                    for g2 in range(4):
                        blk = s["Cbar"][4 * g:4 * g + 4, 4 * g2:4 * g2 + 4]
                        Kg[np.ix_(dofs, dofs)] += etas[bs[g]] * Bg.T @ blk @ Bmat(bs[g2])
            if fext is not None:
                Rg -= (k / n_steps) * np.asarray(fext).ravel()
                Rc -= (k / n_steps) * np.asarray(fext).ravel()
            rnorm = np.linalg.norm(Rg[free])
            if record is not None:
                record.append((k, it, rnorm, rmic))
            if rnorm < tol_macro and rmic < tol_micro:
                iters.append(it)
                break
            if not rnorm < 1e10:
                raise RuntimeError("macro residual above 1e10: Newton diverged")
            dq = np.zeros(2 * nnode)
            dq[free] = np.linalg.solve(Kg[np.ix_(free, free)], -Rc[free])
            q = q + dq.reshape(nnode, 2)
            for e in range(nel):
                Fbs, wq, s = sols[e]
                upd = s["x_r"].copy()
                for g in range(4):
                    dF = dq.reshape(nnode, 2)[conn[e]].T @ grads[4 * e + g]
                    upd += wq[g] * (s["X_M"][g] @ dF.ravel())
                ws[e] = ws[e] - upd
        else:
            raise RuntimeError("macro Newton did not converge")
    out = []
    for e in range(nel):
        Fbs, wq, s = sols[e]
        out.append(dict(Fbar=np.array(Fbs), Pbar=s["Pbar"], Cbar=s["Cbar"], sigma_eff=s["sigma_eff"], w=ws[e]))
    return out, iters, q


def staggered_fe2(macro, rves, F_final, n_steps=1, tol_macro=1e-9, tol_micro=1e-12,
                  maxit=25, maxit_micro=50, record=None, fext=None, micro_start="predicted",
                  micro_record=None):
    """Classical (staggered, nested) FE^2 of Section 4.1 on the same macro
    problem as ``monolithic_fe2``: in every macro Newton iteration each RVE is
    first brought to micro equilibrium r_m = 0 at its current Fbar by an inner
    Newton (starting from its last state), then Pbar and the condensed tangent
    Cbar = (K_MM - K_Mm K_mm^-1 K_mM)/|Omega| at that equilibrium give the
    macro residual and stiffness (Eq. (solution1)).  After the macro update
    the micro states follow Eq. (reduction), dw~ = -L^-1 E dq = -X_M : dFbar,
    and are re-equilibrated in the next iteration.
    ``fext`` as in monolithic_fe2.  ``micro_start`` = "last_converged" starts
    every inner Newton from the micro states of the last converged load step
    instead (no Eq. (reduction) update): the reading of Section 5.2, Table 2,
    whose RVE residual sequences at macro iterations 3 and 4 of load step 1
    coincide.  ``micro_record`` (a list) receives (step, it, max_b ||r_m||)
    before every inner update.  Returns the converged per-Gauss-point
    states, the macro iteration count of every load step, the total number of
    inner micro iterations and q."""
    X, conn, bnd = macro
    grads, etas, _ = macro_gauss(X, conn)
    nb = len(etas)
    nnode = len(X)
    q = X.copy()
    ws = [np.zeros(2 * (r["N"] ** 2 - 1)) for r in rves]
    free = np.ones(2 * nnode, bool)
    for n in bnd:
        free[2 * n:2 * n + 2] = False
    iters, micro_total = [], 0
    w_conv = [w.copy() for w in ws]
    for k in range(1, n_steps + 1):
        Fk = np.eye(2) + (k / n_steps) * (np.asarray(F_final) - np.eye(2))
        q[bnd] = X[bnd] @ Fk.T
        for it in range(maxit):
            Kg = np.zeros((2 * nnode, 2 * nnode))
            Rg = np.zeros(2 * nnode)
            sols = []
            hist = []
            for b in range(nb):
                e = b // 4
                Fb = q[conn[e]].T @ grads[b]
                r = rves[b]
                if micro_start == "last_converged":
                    ws[b] = w_conv[b].copy()
                ws[b], mit = micro_equilibrate(r["N"], 2, r["phase"], r["mat"], Fb, ws[b], tol=tol_micro,
                                               maxit=maxit_micro, history=hist)
                micro_total += mit
                s = rve_solve(r["N"], 2, r["phase"], r["mat"], Fb, ws[b])
                sols.append((Fb, s))
                Bm = np.zeros((4, 8))
                for A_ in range(4):
                    for i in range(2):
                        for J in range(2):
                            Bm[2 * i + J, 2 * A_ + i] = grads[b][A_, J]
                dofs = np.array([[2 * conn[e][A_], 2 * conn[e][A_] + 1] for A_ in range(4)]).ravel()
                Kg[np.ix_(dofs, dofs)] += etas[b] * Bm.T @ s["Cbar"] @ Bm
                Rg[dofs] += etas[b] * Bm.T @ s["Pbar"].ravel()
            if fext is not None:
                Rg -= (k / n_steps) * np.asarray(fext).ravel()
            rnorm = np.linalg.norm(Rg[free])
            if record is not None:
                record.append((k, it, rnorm))
            if micro_record is not None:
                # the largest residual over the RVEs before each inner update
                for j in range(max(len(h) for h in hist)):
                    micro_record.append((k, it, max(h[j] for h in hist if j < len(h))))
            if rnorm < tol_macro:
                iters.append(it)
                w_conv = [w.copy() for w in ws]
                break
            if not rnorm < 1e10:
                raise RuntimeError("macro residual above 1e10: Newton diverged")
            dq = np.zeros(2 * nnode)
            dq[free] = np.linalg.solve(Kg[np.ix_(free, free)], -Rg[free])
            q = q + dq.reshape(nnode, 2)
            if micro_start == "last_converged":
                continue
            # Eq. (reduction): dw~ = -L^-1 E dq, i.e. -X_M : dFbar per Gauss point
            for b in range(nb):
                e = b // 4
                dF = dq.reshape(nnode, 2)[conn[e]].T @ grads[b]
                ws[b] = ws[b] - sols[b][1]["X_M"] @ dF.ravel()
        else:
            raise RuntimeError("macro Newton did not converge")
    out = []
    for b in range(nb):
        Fb, s = sols[b]
        out.append(dict(Fbar=Fb, Pbar=s["Pbar"], Cbar=s["Cbar"], sigma_eff=s["sigma_eff"], w=ws[b]))
    return out, iters, micro_total, q


# ---------------------------------------------------------------------------
# relative-error convention used by every parity check
# ---------------------------------------------------------------------------
def rel_err(x, ref, floor=0.0):
    x = np.asarray(x, float)
    ref = np.asarray(ref, float)
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), floor, 1e-300))
