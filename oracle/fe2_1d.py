"""FP64 CPU oracle of the 1+1-dimensional convergence study (Section 5.1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` may import this module.  It shares
no code with the CUDA path and never imports the product package.

What it computes (Hesch, Schmidt & Schuss, arXiv 2312.12771, Section 5.1):

* the macro bar B0 = (0, 1000) and the RVE (0, 1) with the strain energy
  Psi~ = lambda(X~) (F~^2 - 1), lambda(X~) = 20 / cos(2 pi X~ / 3 - pi / 3),
  body load B = 1, phi(0) = 0, phi(1000) = 37575 sqrt(3) / (2 pi), and
  w~ = 0 at both ends of the RVE (Eq. (Con)(ii));
* the two printed weak forms of that section (the macro equation with the
  load 1/2 int delta phi, the micro equation with zero right-hand side), on
  2^k linear macro elements times 2^k linear micro elements, with three
  approximations of w~ in the macro direction X:
    basis "1"     continuous bilinear in (X, X~)                  p = [1, 1]
    basis "0"     piecewise constant per macro element            p = [0, 1]
                  (Section 3, Eqs. (constSolution1), (constSolution2))
    basis "delta" one micro field per macro Gauss point (Dirac)   p = [delta, 1]
                  (Section 3, Eqs. (fluctVaria_dirac), (fluctSolution))
  assembled as one symmetric linear system and solved with a sparse direct
  solver (library primitive);
* the analytic solutions Eqs. (sol1D_phi), (sol1D_wt) and the relative L2
  errors err_phi, err_w of the section.

The problem is linear in (phi, w~): the stress of Psi~ is 2 lambda F~ and the
printed weak forms are that stress balance divided by 2.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse
import scipy.sparse.linalg

LENGTH = 1000.0
PHI_RIGHT = 37575.0 * math.sqrt(3.0) / (2.0 * math.pi)
BASES = ("1", "0", "delta")


def lam(Xt):
    """lambda(X~) = 20 [cos(2 pi X~ / 3 - pi / 3)]^-1 (Section 5.1)."""
    return 20.0 / np.cos(2.0 * np.pi / 3.0 * Xt - np.pi / 3.0)


def phi_exact(X):
    """Eq. (sol1D_phi)."""
    s3 = math.sqrt(3.0)
    return -3.0 * s3 / (160.0 * math.pi) * X ** 2 + 3003.0 * s3 / (80.0 * math.pi) * X


def F_exact(X):
    """F^a = d phi^a / dX."""
    s3 = math.sqrt(3.0)
    return -3.0 * s3 / (80.0 * math.pi) * X + 3003.0 * s3 / (80.0 * math.pi)


def w_exact(X, Xt):
    """Eq. (sol1D_wt)."""
    return F_exact(X) * (np.sin(2.0 * np.pi / 3.0 * Xt - np.pi / 3.0) / math.sqrt(3.0) - Xt + 0.5)


def _gauss(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w          # on (0, 1)


def solve(k, basis, ngx=2, ngy=5):
    """FE solution on 2^k x 2^k elements.  Returns dict(phi [n+1] nodal values,
    w [n_w][m+1] nodal micro values of every w~ function (row per macro node,
    element or Gauss point), K, basis, n, m, ngx)."""
    if basis not in BASES:
        raise ValueError(basis)
    n = m = 2 ** k
    h, g = LENGTH / n, 1.0 / m
    xg, wgx = _gauss(ngx)
    yg, wgy = _gauss(ngy)
    nrow = {"1": n + 1, "0": n, "delta": n * ngx}[basis]
    nphi = n + 1
    ndof = nphi + nrow * (m - 1)

    def wdof(row, c):
        # micro node c of w~ row `row`; the end nodes c = 0, m are fixed at zero
        return np.where((c >= 1) & (c <= m - 1), nphi + row * (m - 1) + (c - 1), -1)

    # every (macro element e, macro point a, micro element f, micro point b)
    e, a, f, b = np.meshgrid(np.arange(n), np.arange(ngx), np.arange(m), np.arange(ngy), indexing="ij")
    e, a, f, b = (v.ravel() for v in (e, a, f, b))
    wt = lam((f + yg[b]) * g) * (h * wgx[a]) * (g * wgy[b])
    Nx = np.stack([1.0 - xg[a], xg[a]])                 # macro hats at X
    dM = np.array([-1.0 / g, 1.0 / g])                   # micro hat slopes in element f
    dofs = [e, e + 1]
    vals = [np.full(e.shape, -1.0 / h), np.full(e.shape, 1.0 / h)]
    for c in range(2):                                    # micro node f + c
        if basis == "1":
            for i in range(2):                            # macro node e + i
                dofs.append(wdof(e + i, f + c))
                vals.append(Nx[i] * dM[c])
        else:
            row = e if basis == "0" else e * ngx + a
            dofs.append(wdof(row, f + c))
            vals.append(np.full(e.shape, dM[c]))
    D = np.stack(dofs)
    V = np.stack(vals)
    rows, cols, data = [], [], []
    for p in range(len(D)):
        for q in range(len(D)):
            ok = (D[p] >= 0) & (D[q] >= 0)
            rows.append(D[p][ok])
            cols.append(D[q][ok])
            data.append((wt * V[p] * V[q])[ok])
    K = scipy.sparse.coo_matrix((np.concatenate(data), (np.concatenate(rows), np.concatenate(cols))),
                                shape=(ndof, ndof)).tocsr()
    rhs = np.zeros(ndof)
    np.add.at(rhs, np.arange(n), 0.5 * h / 2.0)          # 1/2 int N_i dX
    np.add.at(rhs, np.arange(1, n + 1), 0.5 * h / 2.0)
    u = np.zeros(ndof)
    u[n] = PHI_RIGHT
    free = np.setdiff1d(np.arange(ndof), [0, n])
    r = rhs - K @ u
    u[free] = scipy.sparse.linalg.spsolve(K[free][:, free].tocsc(), r[free])
    W = np.zeros((nrow, m + 1))
    W[:, 1:m] = u[nphi:].reshape(nrow, m - 1)
    return dict(phi=u[:nphi], w=W, K=K, basis=basis, n=n, m=m, ngx=ngx)


def _w_rows_at(sol, e, xi):
    """w~ nodal values (over X~) at local macro coordinate xi of element e."""
    W, basis = sol["w"], sol["basis"]
    if basis == "1":
        return (1.0 - xi)[:, None] * W[e] + xi[:, None] * W[e + 1]
    if basis == "0":
        return W[e]
    # Dirac: the field of Gauss point j holds on the j-th part of the element,
    # the parts being the Gauss weights laid end to end
    ngx = sol["ngx"]
    _, wgx = _gauss(ngx)
    edges = np.concatenate([[0.0], np.cumsum(wgx)])
    j = np.clip(np.searchsorted(edges, xi, side="right") - 1, 0, ngx - 1)
    return W[e * ngx + j]


def errors(sol, nq=4):
    """Relative L2 errors err_phi (over B0) and err_w (over B0 x RVE), each
    macro element split at the Gauss-weight boundaries so that the Dirac
    field is integrated piece by piece."""
    n, m = sol["n"], sol["m"]
    h, g = LENGTH / n, 1.0 / m
    ngx = sol["ngx"]
    _, wgx = _gauss(ngx)
    edges = np.concatenate([[0.0], np.cumsum(wgx)])
    xq, wq = _gauss(nq)
    yq, wyq = _gauss(nq + 2)
    num_p = den_p = num_w = den_w = 0.0
    for s in range(ngx):                                  # parts of each element
        xi = edges[s] + (edges[s + 1] - edges[s]) * xq
        wx = (edges[s + 1] - edges[s]) * wq * h
        for e in range(n):
            X = (e + xi) * h
            ph = (1.0 - xi) * sol["phi"][e] + xi * sol["phi"][e + 1]
            pa = phi_exact(X)
            num_p += np.sum(wx * (ph - pa) ** 2)
            den_p += np.sum(wx * pa ** 2)
            Wr = np.broadcast_to(_w_rows_at(sol, e, xi), (len(xi), m + 1))
            for f in range(m):
                Xt = (f + yq) * g
                wh = (1.0 - yq)[None, :] * Wr[:, f:f + 1] + yq[None, :] * Wr[:, f + 1:f + 2]
                wa = w_exact(X[:, None], Xt[None, :])
                ww = wx[:, None] * (g * wyq)[None, :]
                num_w += np.sum(ww * (wh - wa) ** 2)
                den_w += np.sum(ww * wa ** 2)
    return math.sqrt(num_p / den_p), math.sqrt(num_w / den_w)


def effective_modulus(m, ngy=5):
    """2 <lambda^-1>^-1 of the micro FE problem on m linear elements: the
    micro stress 2 lambda (F + w~') per unit macro gradient F, which is
    constant along the RVE at micro equilibrium (zero-end fluctuation)."""
    g = 1.0 / m
    yg, wgy = _gauss(ngy)
    # element stiffness int lambda over each element (per unit slope squared)
    kel = np.array([np.sum(lam((f + yg) * g) * g * wgy) for f in range(m)]) / g ** 2
    # condensed micro problem: the slopes s_f = F + w~'_f satisfy kel_f g s_f = c
    # for one constant c, and sum_f g s_f = F  =>  c = F / sum_f (1 / kel_f)
    c_per_F = 1.0 / np.sum(1.0 / kel)
    return 2.0 * c_per_F
