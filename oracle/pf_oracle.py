"""FP64 CPU oracle for the pressurised AT2 phase-field functional and RMTR.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this module.  The CUDA
library never calls it and shares no code with it.

Everything here is plain float64 numpy written from the paper:

* the functional, Sec. 2 eq. (pressurized) with the AT2 choices
  g(c)=(1-c)^2, w(c)=c^2, c_w=2 (Sec. 2.1), discretised with Q1 Lagrange
  elements (Sec. 2.2) on a uniform structured grid, 2^d-point Gauss rule;
* its gradient and Hessian (derived by hand, written out below);
* the level hierarchy and transfer operators I, R=I^T, P (Sec. 3);
* the level objective h^l of eq. (second_order_consistency) with the terms of
  eq. (delta_terms), the V-cycle of Algorithm 1, the trust-region method of
  Algorithm 2, Convergence_control of Algorithm 3, the ratios of
  eq. (rho_tr) and eq. (rho_ml), and Hessian lagging (Sec. 4.2.1);
* the trust-region subproblem eq. (model_qp), solved by a projected
  truncated CG (the default reading), or by the paper's own QP solvers
  (Sec. 4.2.2): multicolour symmetric projected Gauss-Seidel smoothing and
  MPRGP on the coarsest level;
* the trust-region gate of a proposed iterate (eq. (rho_tr) with
  Algorithm 3's acceptance), used by the learned initial iterate.

Readings where the paper is silent or inconsistent (all listed in the design
notes): the sign of the pressure term (+p g(c) div u, derived from eq.
(energy_not_reg) and eq. (traction_forces), the printed eq. (pressurized)
has the opposite sign); the quadrature rule; l_s = 2 h_finest on all levels;
the projection P = diag(R 1)^-1 R; the coarse feasible set by max/min over
the prolongation support; the TR constants; the subproblem solver.

Layout: a state vector x holds (d+1) planes [u_x, u_y, (u_z), c], each of
N = prod(n) nodal values in lexicographic order with x fastest.
Level index 0 is the coarsest level (the paper's l = 1).

Parity status:
* energy, gradient and hessvec: the patch test, exact 5-point finite
  differences, symmetry and an independently assembled dense Hessian; the
  exact quartic energy difference against the polynomial it must be;
* the Jacobi diagonal: that dense Hessian's diagonal;
* Convergence_control: a hand-written table of Algorithm 3's cases;
* transfers: linear reproduction, adjointness and the coarse feasible set's
  defining property;
* rasterisation: lattice-point counts of discs and plates, the centred
  crack's three rows, the paper's printed dof counts for the grids;
* the subproblem: 1D and separable closed forms, the bent Cauchy path, the
  radius cap; PGS and MPRGP: the exact one-sweep diagonal case, the KKT
  point, the 1D closed form;
* the gate: the ratio from the exact quartic within the cancellation bound;
* the solver: the 1D closed-form phase-field profile, Sneddon's opening and
  the invariants, and the onset of propagation at the Griffith pressure;
* planted mistakes (a sign, a dropped pressure term, a model sign, the
  projection, the diagonal, swapped radius factors or thresholds, the gate's
  sign, an unprojected Gauss-Seidel step, MPRGP's gradient sign) each fail a
  named test.
The level model's choice of f~^l beyond "the same functional on the coarse
grid" is "parity unpinned" apart from its coherence identities.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

LINE2D = 0
DISC3D = 1
BOX3D = 2

GALERKIN = 0
FIRST_ORDER = 1


# --------------------------------------------------------------------------
# material and grid
# --------------------------------------------------------------------------
@dataclass
class Params:
    """Material/load parameters of eq. (pressurized) (Sec. 2)."""
    E: float = 1.0
    nu: float = 0.3
    Gc: float = 1.0
    ls: float = 0.03125
    p: float = 0.0
    k_res: float = 0.0  # residual stiffness; the paper has none (0)

    @property
    def lam(self) -> float:
        return self.E * self.nu / ((1.0 + self.nu) * (1.0 - 2.0 * self.nu))

    @property
    def mu(self) -> float:
        return self.E / (2.0 * (1.0 + self.nu))


class Grid:
    """Uniform Q1 grid: n[k] nodes along axis k, spacing h, origin 0."""

    def __init__(self, dim: int, n, h: float):
        self.dim = dim
        self.n = tuple(int(v) for v in n)[:dim]
        self.h = float(h)
        self.N = int(np.prod(self.n))
        self.ne = tuple(v - 1 for v in self.n)
        self.NE = int(np.prod(self.ne))
        # corner a = a_x + 2 a_y + 4 a_z ; quadrature point q likewise
        self.corners = [tuple((a >> k) & 1 for k in range(dim)) for a in range(2 ** dim)]
        self._tables()

    def node_index(self, idx):
        """Lexicographic node number (x fastest) of integer coordinates."""
        out = 0
        stride = 1
        for k in range(self.dim):
            out = out + idx[k] * stride
            stride *= self.n[k]
        return out

    def node_coords(self):
        """Integer coordinates of all nodes, shape (dim, N)."""
        rev = np.unravel_index(np.arange(self.N), self.n[::-1])
        return np.stack(rev[::-1])

    def element_connectivity(self, elems=None) -> np.ndarray:
        """(E, 2^d) node numbers of each element's corners."""
        if elems is None:
            elems = np.arange(self.NE)
        elems = np.asarray(elems, dtype=np.int64)
        eidx = []
        rem = elems.copy()
        for k in range(self.dim):
            eidx.append(rem % self.ne[k])
            rem //= self.ne[k]
        conn = np.empty((len(elems), 2 ** self.dim), dtype=np.int64)
        for a, off in enumerate(self.corners):
            conn[:, a] = self.node_index([eidx[k] + off[k] for k in range(self.dim)])
        return conn

    def elements_touching(self, nodes) -> np.ndarray:
        """All elements that have one of ``nodes`` as a corner."""
        nodes = np.asarray(nodes, dtype=np.int64)
        nidx = []
        rem = nodes.copy()
        for k in range(self.dim):
            nidx.append(rem % self.n[k])
            rem //= self.n[k]
        found = []
        for off in itertools.product([0, 1], repeat=self.dim):
            e = [nidx[k] - off[k] for k in range(self.dim)]
            ok = np.ones(len(nodes), dtype=bool)
            for k in range(self.dim):
                ok &= (e[k] >= 0) & (e[k] < self.ne[k])
            lin = np.zeros(len(nodes), dtype=np.int64)
            stride = 1
            for k in range(self.dim):
                lin = lin + e[k] * stride
                stride *= self.ne[k]
            found.append(lin[ok])
        return np.unique(np.concatenate(found))

    def _tables(self):
        """Q1 shape values / gradients at the 2^d Gauss points of a cell."""
        d, h = self.dim, self.h
        g = 1.0 / math.sqrt(3.0)
        xi = np.array([0.5 * (1.0 - g), 0.5 * (1.0 + g)])  # on [0, 1]
        n1 = np.array([[1.0 - xi[0], xi[0]], [1.0 - xi[1], xi[1]]])  # n1[q, a]
        d1 = np.array([-1.0, 1.0]) / h  # d phi_a / dx along the axis
        Q = 2 ** d
        self.Nq = np.zeros((Q, Q))
        self.dNq = np.zeros((Q, Q, d))
        for q in range(Q):
            qc = [(q >> k) & 1 for k in range(d)]
            for a in range(Q):
                ac = self.corners[a]
                val = 1.0
                for k in range(d):
                    val *= n1[qc[k], ac[k]]
                self.Nq[q, a] = val
                for k in range(d):
                    dv = d1[ac[k]]
                    for m in range(d):
                        if m != k:
                            dv *= n1[qc[m], ac[m]]
                    self.dNq[q, a, k] = dv
        self.wq = (h ** d) / Q  # each Gauss weight times det J

    def boundary_nodes(self) -> np.ndarray:
        ij = self.node_coords()
        on = np.zeros(self.N, dtype=bool)
        for k in range(self.dim):
            on |= (ij[k] == 0) | (ij[k] == self.n[k] - 1)
        return on


def lame(prm: Params):
    return prm.lam, prm.mu


# --------------------------------------------------------------------------
# fracture rasterisation (Sec. 5: nodal c = 1 inside the regularised band)
# --------------------------------------------------------------------------
def rasterize(grid: Grid, kind: int, rows: np.ndarray, band_half_width: float) -> np.ndarray:
    """c = 1 at nodes whose distance to the fracture's mid-surface is <= w/2
    and whose in-surface coordinate lies inside the fracture, else 0
    (Sec. 5 initialisation, band width w = 2h of Sec. 5.2).  Union over
    fractures.  Node coordinates are i*h."""
    ij = grid.node_coords().astype(np.float64) * grid.h
    c = np.zeros(grid.N)
    rows = np.atleast_2d(np.asarray(rows, dtype=np.float64))
    for r in rows:
        if kind == LINE2D:
            cx, cy, th, a = r
            t = np.array([math.cos(th), math.sin(th)])
            nrm = np.array([-math.sin(th), math.cos(th)])
            dx = ij[0] - cx
            dy = ij[1] - cy
            dn = np.abs(nrm[0] * dx + nrm[1] * dy)
            dt = np.abs(t[0] * dx + t[1] * dy)
            inside = (dn <= band_half_width) & (dt <= a)
        elif kind == DISC3D:
            cen = r[0:3]
            nv = r[3:6]
            rad = r[6]
            dx = ij[0] - cen[0]
            dy = ij[1] - cen[1]
            dz = ij[2] - cen[2]
            dn = nv[0] * dx + nv[1] * dy + nv[2] * dz
            px = dx - dn * nv[0]
            py = dy - dn * nv[1]
            pz = dz - dn * nv[2]
            inside = (np.abs(dn) <= band_half_width) & (px * px + py * py + pz * pz <= rad * rad)
        elif kind == BOX3D:
            # a rectangular plate: centre, unit normal n, unit in-plane axes
            # a and b, half-lengths along a and b (the "smooth
            # parallelepipeds" of Sec. 5.2 are these plates widened to the
            # band)
            cen, nv, av, bv = r[0:3], r[3:6], r[6:9], r[9:12]
            ha, hb = r[12], r[13]
            dx = ij[0] - cen[0]
            dy = ij[1] - cen[1]
            dz = ij[2] - cen[2]
            dn = nv[0] * dx + nv[1] * dy + nv[2] * dz
            da = av[0] * dx + av[1] * dy + av[2] * dz
            db = bv[0] * dx + bv[1] * dy + bv[2] * dz
            inside = (np.abs(dn) <= band_half_width) & (np.abs(da) <= ha) & (np.abs(db) <= hb)
        else:
            raise ValueError("unknown fracture kind")
        c[inside] = 1.0
    return c


# --------------------------------------------------------------------------
# functional, gradient, Hessian (eq. pressurized with AT2; Q1, Gauss 2^d)
# --------------------------------------------------------------------------
def _split(grid: Grid, x):
    d, N = grid.dim, grid.N
    return x[: d * N].reshape(d, N), x[d * N:]


def _chunks(grid: Grid, elems, size=1 << 16):
    if elems is None:
        elems = np.arange(grid.NE)
    for s in range(0, len(elems), size):
        yield elems[s: s + size]


def _qp_state(grid: Grid, conn, U, C):
    """Displacement gradient, phase field and its gradient at the Gauss points."""
    Ue = U[:, conn]  # (d, E, A)
    Ce = C[conn]  # (E, A)
    G = np.einsum("qak,iea->eqik", grid.dNq, Ue, optimize=True)  # G[e,q,i,k] = d u_i / d x_k
    c = np.einsum("qa,ea->eq", grid.Nq, Ce, optimize=True)
    gc = np.einsum("qak,ea->eqk", grid.dNq, Ce, optimize=True)
    return G, c, gc


def _degradation(prm: Params, c):
    """g(c) = (1-k)(1-c)^2 + k and its first two derivatives (AT2, Sec. 2.1)."""
    k = prm.k_res
    g = (1.0 - k) * (1.0 - c) ** 2 + k
    dg = -2.0 * (1.0 - k) * (1.0 - c)
    ddg = 2.0 * (1.0 - k) * np.ones_like(c)
    return g, dg, ddg


def _strain_terms(prm: Params, G):
    lam, mu = lame(prm)
    d = G.shape[-1]
    eps = 0.5 * (G + np.swapaxes(G, -1, -2))
    tr = np.trace(G, axis1=-2, axis2=-1)
    psi = 0.5 * lam * tr ** 2 + mu * np.sum(eps * eps, axis=(-2, -1))
    sig = 2.0 * mu * eps + lam * tr[..., None, None] * np.eye(d)
    return eps, tr, psi, sig


def energy(grid: Grid, prm: Params, x, elems=None) -> float:
    """E(u,c) = sum_e sum_q w [ g(c) psi(eps(u)) + Gc/2 (c^2/ls + ls |grad c|^2)
    + p g(c) div u ]  (eq. pressurized with the sign reading, AT2)."""
    U, C = _split(grid, x)
    total = 0.0
    for ch in _chunks(grid, elems):
        conn = grid.element_connectivity(ch)
        G, c, gc = _qp_state(grid, conn, U, C)
        _, tr, psi, _ = _strain_terms(prm, G)
        g, _, _ = _degradation(prm, c)
        dens = g * psi + 0.5 * prm.Gc * (c * c / prm.ls + prm.ls * np.sum(gc * gc, axis=-1)) \
            + prm.p * g * tr
        total += grid.wq * float(np.sum(dens))
    return total


def energy_diff_coeffs(grid: Grid, prm: Params, x, s, elems=None) -> np.ndarray:
    """Coefficients a1..a4 of E(x + t s) - E(x) = a1 t + a2 t^2 + a3 t^3 + a4 t^4.

    Along a line the discrete functional is a quartic polynomial in t (the
    density is a polynomial of degree 4 in the nodal values and the
    quadrature is a finite sum), so the actual reduction E(x) - E(x+s) used
    by the trust-region ratios eq. (rho_tr) / eq. (rho_ml) equals
    -(a1 + a2 + a3 + a4) exactly.  Each coefficient is summed from per-point
    products of small quantities, so it keeps its relative accuracy when the
    reduction is far below the round-off of E itself."""
    U, C = _split(grid, x)
    SU, SC = _split(grid, s)
    lam, mu = lame(prm)
    k = prm.k_res
    out = np.zeros(4)
    for ch in _chunks(grid, elems):
        conn = grid.element_connectivity(ch)
        G, c, gc = _qp_state(grid, conn, U, C)
        Gs, sc, gsc = _qp_state(grid, conn, SU, SC)
        eps, tr, psi0, _ = _strain_terms(prm, G)
        epss, trs, psi2, _ = _strain_terms(prm, Gs)
        psi1 = lam * tr * trs + 2.0 * mu * np.sum(eps * epss, axis=(-2, -1))
        g0 = (1.0 - k) * (1.0 - c) ** 2 + k
        g1 = -2.0 * (1.0 - k) * (1.0 - c) * sc
        g2 = (1.0 - k) * sc * sc
        p = prm.p
        # g(t) psi(t) + p g(t) (tr + t trs) + Gc/2 (c(t)^2/ls + ls |grad c(t)|^2)
        a1 = g0 * psi1 + g1 * psi0 + p * (g0 * trs + g1 * tr) \
            + prm.Gc * (c * sc / prm.ls + prm.ls * np.sum(gc * gsc, axis=-1))
        a2 = g0 * psi2 + g1 * psi1 + g2 * psi0 + p * (g1 * trs + g2 * tr) \
            + 0.5 * prm.Gc * (sc * sc / prm.ls + prm.ls * np.sum(gsc * gsc, axis=-1))
        a3 = g1 * psi2 + g2 * psi1 + p * g2 * trs
        a4 = g2 * psi2
        out += grid.wq * np.array([np.sum(a1), np.sum(a2), np.sum(a3), np.sum(a4)])
    return out


def energy_diff(grid: Grid, prm: Params, x, s, elems=None) -> float:
    """E(x + s) - E(x) from the quartic coefficients."""
    a = energy_diff_coeffs(grid, prm, x, s, elems)
    return float(a[0] + a[1] + a[2] + a[3])


def _scatter(grid: Grid, conn, contrib_u, contrib_c, out):
    """out[plane i, node] += element contributions (owner-free sum)."""
    d, N = grid.dim, grid.N
    idx = conn.ravel()
    for i in range(d):
        out[i * N:(i + 1) * N] += np.bincount(idx, weights=contrib_u[i].ravel(), minlength=N)
    out[d * N:] += np.bincount(idx, weights=contrib_c.ravel(), minlength=N)


def gradient(grid: Grid, prm: Params, x, elems=None) -> np.ndarray:
    """dE/dx.  u-rows: int g (sigma(u) + p I) : grad phi ;
    c-rows: int [g'(psi + p div u) + Gc c/ls] phi + Gc ls grad c . grad phi."""
    U, C = _split(grid, x)
    out = np.zeros_like(x)
    d = grid.dim
    for ch in _chunks(grid, elems):
        conn = grid.element_connectivity(ch)
        G, c, gc = _qp_state(grid, conn, U, C)
        _, tr, psi, sig = _strain_terms(prm, G)
        g, dg, _ = _degradation(prm, c)
        S = g[..., None, None] * (sig + prm.p * np.eye(d))  # (E,Q,d,d)
        cu = grid.wq * np.einsum("eqik,qak->iea", S, grid.dNq, optimize=True)
        s0 = dg * (psi + prm.p * tr) + prm.Gc * c / prm.ls
        s1 = prm.Gc * prm.ls * gc
        cc = grid.wq * (np.einsum("eq,qa->ea", s0, grid.Nq, optimize=True) + np.einsum("eqk,qak->ea", s1, grid.dNq, optimize=True))
        _scatter(grid, conn, cu, cc, out)
    return out


def hessvec(grid: Grid, prm: Params, x, v, elems=None) -> np.ndarray:
    """Hessian of E at x applied to v (second derivatives written out):
    uu: g sigma(v_u) : grad phi
    uc: g' v_c (sigma(u) + p I) : grad phi
    cu: g' (sigma(u) : eps(v_u) + p div v_u) phi
    cc: (g''(psi + p div u) + Gc/ls) v_c phi + Gc ls grad v_c . grad phi."""
    U, C = _split(grid, x)
    V, VC = _split(grid, v)
    out = np.zeros_like(x)
    d = grid.dim
    for ch in _chunks(grid, elems):
        conn = grid.element_connectivity(ch)
        G, c, _ = _qp_state(grid, conn, U, C)
        Gv, vc, gvc = _qp_state(grid, conn, V, VC)
        _, tr, psi, sig = _strain_terms(prm, G)
        epsv, trv, _, sigv = _strain_terms(prm, Gv)
        g, dg, ddg = _degradation(prm, c)
        T = sig + prm.p * np.eye(d)
        S = g[..., None, None] * sigv + (dg * vc)[..., None, None] * T
        cu = grid.wq * np.einsum("eqik,qak->iea", S, grid.dNq, optimize=True)
        s0 = dg * np.sum(T * epsv, axis=(-2, -1)) + (ddg * (psi + prm.p * tr) + prm.Gc / prm.ls) * vc
        s1 = prm.Gc * prm.ls * gvc
        cc = grid.wq * (np.einsum("eq,qa->ea", s0, grid.Nq, optimize=True) + np.einsum("eqk,qak->ea", s1, grid.dNq, optimize=True))
        _scatter(grid, conn, cu, cc, out)
    return out


def hess_diag(grid: Grid, prm: Params, x, elems=None) -> np.ndarray:
    """Diagonal of the Hessian of E at x (the Jacobi preconditioner of the
    subproblem CG): for a u_i dof of corner a,
    g [lam (d_i phi_a)^2 + mu (|grad phi_a|^2 + (d_i phi_a)^2)]; for a c dof,
    (g''(psi + p div u) + Gc/ls) phi_a^2 + Gc ls |grad phi_a|^2."""
    U, C = _split(grid, x)
    out = np.zeros_like(x)
    lam, mu = lame(prm)
    d = grid.dim
    dn2 = grid.dNq ** 2  # (Q, A, d)
    gn2 = np.sum(dn2, axis=-1)  # (Q, A)
    for ch in _chunks(grid, elems):
        conn = grid.element_connectivity(ch)
        G, c, _ = _qp_state(grid, conn, U, C)
        _, tr, psi, _ = _strain_terms(prm, G)
        g, _, ddg = _degradation(prm, c)
        cu = np.stack([grid.wq * np.einsum("eq,qa->ea", g, lam * dn2[:, :, i] + mu * (gn2 + dn2[:, :, i]),
                                           optimize=True) for i in range(d)])
        m = ddg * (psi + prm.p * tr) + prm.Gc / prm.ls
        cc = grid.wq * (np.einsum("eq,qa->ea", m, grid.Nq ** 2, optimize=True)
                        + prm.Gc * prm.ls * np.sum(gn2, axis=0)[None, :])
        _scatter(grid, conn, cu, cc, out)
    return out


def dense_hessian(grid: Grid, prm: Params, x) -> np.ndarray:
    """Independent assembly of the full Hessian from element matrices built
    basis pair by basis pair (loops; tiny meshes only)."""
    d, N = grid.dim, grid.N
    lam, mu = lame(prm)
    U, C = _split(grid, x)
    nd = (d + 1) * N
    H = np.zeros((nd, nd))
    conn_all = grid.element_connectivity()
    A = 2 ** d
    for e in range(grid.NE):
        conn = conn_all[e]
        for q in range(A):
            w = grid.wq
            phi = grid.Nq[q]
            dphi = grid.dNq[q]  # (A, d)
            c = float(phi @ C[conn])
            Gu = np.array([[float(dphi[:, k] @ U[i, conn]) for k in range(d)] for i in range(d)])
            eps = 0.5 * (Gu + Gu.T)
            tr = float(np.trace(Gu))
            psi = 0.5 * lam * tr * tr + mu * float(np.sum(eps * eps))
            sig = 2 * mu * eps + lam * tr * np.eye(d)
            kk = prm.k_res
            g = (1 - kk) * (1 - c) ** 2 + kk
            dg = -2 * (1 - kk) * (1 - c)
            ddg = 2 * (1 - kk)
            for a in range(A):
                for b in range(A):
                    # u-u block
                    for i in range(d):
                        for j in range(d):
                            val = lam * dphi[a, i] * dphi[b, j] + mu * dphi[a, j] * dphi[b, i]
                            if i == j:
                                val += mu * float(dphi[a] @ dphi[b])
                            H[i * N + conn[a], j * N + conn[b]] += w * g * val
                    # u-c and c-u blocks
                    for i in range(d):
                        val = dg * (float(sig[i] @ dphi[a]) + prm.p * dphi[a, i]) * phi[b]
                        H[i * N + conn[a], d * N + conn[b]] += w * val
                        H[d * N + conn[b], i * N + conn[a]] += w * val
                    # c-c block
                    val = (ddg * (psi + prm.p * tr) + prm.Gc / prm.ls) * phi[a] * phi[b] \
                        + prm.Gc * prm.ls * float(dphi[a] @ dphi[b])
                    H[d * N + conn[a], d * N + conn[b]] += w * val
    return H


# --------------------------------------------------------------------------
# hierarchy and transfers (Sec. 3: I^l, R^l = (I^l)^T, P^l)
# --------------------------------------------------------------------------
def _prolong_1d(nc: int) -> sp.csr_matrix:
    nf = 2 * nc - 1
    rows, cols, vals = [], [], []
    for i in range(nc):
        rows.append(2 * i); cols.append(i); vals.append(1.0)
    for i in range(nc - 1):
        rows += [2 * i + 1, 2 * i + 1]; cols += [i, i + 1]; vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def prolongation_matrix(coarse: Grid) -> sp.csr_matrix:
    """Q1 nodal interpolation from a coarse grid to its 2:1 refinement
    (tensor product of the 1D [1/2, 1, 1/2] rule, x fastest)."""
    M = None
    for k in range(coarse.dim):
        m1 = _prolong_1d(coarse.n[k])
        M = m1 if M is None else sp.kron(m1, M, format="csr")
    return M.tocsr()


class Transfer:
    """I (coarse->fine), R = I^T, P = diag(R 1)^-1 R, and the support max/min
    used to build the coarse feasible set."""

    def __init__(self, coarse: Grid, fine: Grid):
        self.coarse, self.fine = coarse, fine
        self.Imat = prolongation_matrix(coarse)
        self.Rmat = self.Imat.T.tocsr()
        rsum = np.asarray(self.Rmat.sum(axis=1)).ravel()
        self.Pmat = sp.diags(1.0 / rsum) @ self.Rmat
        self.Pmat = self.Pmat.tocsr()
        Ic = self.Imat.tocsc()
        Ic.sort_indices()
        self._colptr = Ic.indptr
        self._rows = Ic.indices
        self.nf = fine.dim + 1

    def _per_plane(self, M, v, n_in, n_out):
        out = np.empty(self.nf * n_out)
        for f in range(self.nf):
            out[f * n_out:(f + 1) * n_out] = M @ v[f * n_in:(f + 1) * n_in]
        return out

    def prolong(self, vc):
        return self._per_plane(self.Imat, vc, self.coarse.N, self.fine.N)

    def restrict(self, vf):
        return self._per_plane(self.Rmat, vf, self.fine.N, self.coarse.N)

    def project(self, xf):
        return self._per_plane(self.Pmat, xf, self.fine.N, self.coarse.N)

    def support_max(self, vf):
        return self._support_reduce(vf, np.maximum)

    def support_min(self, vf):
        return self._support_reduce(vf, np.minimum)

    def _support_reduce(self, vf, op):
        Nc, Nf = self.coarse.N, self.fine.N
        out = np.empty(self.nf * Nc)
        for f in range(self.nf):
            plane = vf[f * Nf:(f + 1) * Nf]
            vals = plane[self._rows]
            out[f * Nc:(f + 1) * Nc] = op.reduceat(vals, self._colptr[:-1])
        return out


def level_sizes(n_coarse, n_levels):
    """n_l = (n_1 - 1) 2^(l-1) + 1 nodes per axis (uniform refinement)."""
    return [tuple((v - 1) * 2 ** l + 1 for v in n_coarse) for l in range(n_levels)]


# --------------------------------------------------------------------------
# trust-region machinery (Algorithms 2 and 3, eq. model_qp, eq. rho_tr)
# --------------------------------------------------------------------------
@dataclass
class TRParams:
    eta1: float = 0.1
    eta2: float = 0.75
    gamma1: float = 0.5
    gamma2: float = 2.0
    delta0: float = 1.0
    delta_max: float = 1.0
    mu1: int = 1
    mu2: int = 1
    coarse_its: int = 10
    cg_fine: int = 50
    cg_smooth: int = 10
    cg_coarse: int = 500
    cauchy_backtracks: int = 30
    cauchy_c: float = 0.01
    max_cycles: int = 200
    rtol: float = 1e-10
    atol: float = 0.0
    coarse_model: int = FIRST_ORDER
    precondition: bool = True   # Jacobi-preconditioned subproblem CG
    max_restarts: int = 1000000  # CG restarts after projected searches, per subproblem
    pg_ref: float = 0.0         # > 0: stopping test relative to this instead of the start
    level_rtol: float = 1e-3    # non-finest levels stop their TR loop once the
                                # level's projected gradient fell by this factor
    qp_solver: int = 0          # 0: projected truncated CG; 1: the paper's QP
                                # solvers (PGS sweeps, MPRGP on the coarsest)
    pgs_sweeps: int = 2         # symmetric PGS sweeps per subproblem


def proj_box(s, lo, hi):
    return np.minimum(np.maximum(s, lo), hi)


def max_step(s, p, lo, hi, free):
    """Largest alpha >= 0 with lo <= s + alpha p <= hi on the free set."""
    amax = np.inf
    pos = free & (p > 0)
    neg = free & (p < 0)
    if np.any(pos):
        amax = min(amax, float(np.min((hi[pos] - s[pos]) / p[pos])))
    if np.any(neg):
        amax = min(amax, float(np.min((lo[neg] - s[neg]) / p[neg])))
    return max(amax, 0.0)


def _model(g, s, Hs):
    return float(g @ s) + 0.5 * float(s @ Hs)


def solve_subproblem(g, Hv, lo, hi, delta, cg_max, tr: TRParams, stats=None, minv=None):
    """Approximate minimiser of m(s) = g.s + 1/2 s.Hs over lo <= s <= hi
    (eq. model_qp: the TR box intersected with the level's feasible set),
    reaching the sufficient decrease the paper asks of its QP solvers:

    1. generalised Cauchy point s = P(-t g), t from the model's curvature
       along the movable part of -g, capped by the TR radius, halved until
       m(s) <= c1 g.s;
    2. repeated: CG on the free set F = {lo < s < hi} for the reduced model,
       stopped on the forcing test, on non-positive curvature or when the CG
       iterate leaves the box; then a projected search
       s <- P(s + beta d), beta = 1, 1/2, ..., accepted on
       m(new) <= m(s) + c1 grad m(s).(new - s).  Repeated while CG was cut
       by the box and iterations remain.
    minv: inverse diagonal preconditioner (0 where the diagonal is not
    positive); None runs plain CG.
    """
    def H(v):
        if stats is not None:
            stats["hessvecs"] += 1
        return Hv(v)

    movable = ((g < 0) & (hi > 0)) | ((g > 0) & (lo < 0))
    if not np.any(movable):
        return np.zeros_like(g)
    gm = np.where(movable, g, 0.0)
    gmax = float(np.max(np.abs(gm)))
    if gmax == 0.0:
        return np.zeros_like(g)
    t = delta / gmax
    curv = float(gm @ H(gm))
    if curv > 0.0:
        t = min(t, float(gm @ gm) / curv)
    ok = False
    s = np.zeros_like(g)
    Hs = None
    for _ in range(tr.cauchy_backtracks + 1):
        s = proj_box(-t * g, lo, hi)
        Hs = H(s)
        gs = float(g @ s)
        if _model(g, s, Hs) <= tr.cauchy_c * gs:
            ok = True
            break
        t *= 0.5
    if not ok:
        return np.zeros_like(g)

    used = 0
    tol = None
    restarts = 0
    while used < cg_max:
        free = (lo < s) & (s < hi)
        grad_m = g + Hs
        r = np.where(free, -grad_m, 0.0)
        rr = float(r @ r)
        if tol is None:
            r0 = math.sqrt(rr)
            tol = min(0.1, math.sqrt(r0)) * r0
        if math.sqrt(rr) <= tol or rr == 0.0:
            break
        # (preconditioned) CG on the free set from w = 0
        w = np.zeros_like(g)
        Hw = np.zeros_like(g)
        z = r * minv if minv is not None else r
        rz = float(r @ z)
        p = z.copy()
        leave = False
        while used < cg_max:
            q = np.where(free, H(p), 0.0)
            used += 1
            if stats is not None:
                stats["cg"] += 1
            kappa = float(p @ q)
            if kappa <= 0.0:
                amax = max_step(s + w, p, lo, hi, free)
                if np.isfinite(amax):
                    w = w + amax * p
                    Hw = Hw + amax * q
                leave = True
                break
            alpha = rz / kappa
            w = w + alpha * p
            Hw = Hw + alpha * q
            r = r - alpha * q
            rr_new = float(r @ r)
            z = r * minv if minv is not None else r
            rz_new = float(r @ z)
            sw = s + w
            if np.any(free & ((sw < lo) | (sw > hi))):
                leave = True
                break
            if math.sqrt(rr_new) <= tol:
                break
            p = z + (rz_new / rz) * p
            rz = rz_new
        if not leave:
            s = s + w
            Hs = Hs + Hw
            break
        # projected search along d = w
        m_s = _model(g, s, Hs)
        beta = 1.0
        accepted = False
        for _ in range(tr.cauchy_backtracks + 1):
            s_new = proj_box(s + beta * w, lo, hi)
            Hs_new = H(s_new)
            if _model(g, s_new, Hs_new) <= m_s + tr.cauchy_c * float(grad_m @ (s_new - s)):
                accepted = True
                break
            beta *= 0.5
        if not accepted:
            break
        s, Hs = s_new, Hs_new
        restarts += 1
        if restarts > tr.max_restarts:
            break
    return proj_box(s, lo, hi)


# --------------------------------------------------------------------------
# the paper's QP solvers for eq. (model_qp) (Sec. 4.2.2): a few sweeps of
# symmetric projected Gauss-Seidel on the non-coarsest levels, MPRGP on the
# coarsest level
# --------------------------------------------------------------------------
def probe_sparse(grid: Grid, Hv) -> sp.csr_matrix:
    """The (3^d-point block) matrix of the linear map Hv, recovered by
    probing: nodes with equal coordinates mod 3 are at least 3 apart, so
    their neighbourhoods do not overlap, and one product per (colour, field)
    gives all their columns."""
    d, N = grid.dim, grid.N
    F = d + 1
    ij = grid.node_coords()
    colour = np.zeros(N, dtype=np.int64)
    for k in range(d):
        colour += (ij[k] % 3) * 3 ** k
    rows, cols, vals = [], [], []
    # neighbours of every node (within one index per axis)
    for c in range(3 ** d):
        nodes = np.where(colour == c)[0]
        for f in range(F):
            v = np.zeros(F * N)
            v[f * N + nodes] = 1.0
            y = Hv(v)
            nz = np.nonzero(y)[0]
            # the node that owns the nonzero y[r]: the colour-c node within
            # one index of r's node on every axis
            rn = nz % N
            rij = ij[:, rn]
            owner = np.zeros(len(nz), dtype=np.int64)
            for k in range(d):
                # the owner's coordinate on axis k is the one of rij-1, rij, rij+1 with the right residue
                want = (c // 3 ** k) % 3
                cand = rij[k] + ((want - rij[k]) % 3 + 1) % 3 - 1
                owner += cand * (np.prod(grid.n[:k]) if k else 1)
            rows.append(nz)
            cols.append(f * N + owner)
            vals.append(y[nz])
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(F * N, F * N))
    return A


def node_parity_colours(grid: Grid) -> np.ndarray:
    """Colour of every node: sum_k (i_k mod 2) 2^k.  Nodes of one colour are
    at least 2 apart on some axis, so no 3^d-point stencil couples them."""
    ij = grid.node_coords()
    col = np.zeros(grid.N, dtype=np.int64)
    for k in range(grid.dim):
        col += (ij[k] % 2) << k
    return col


def pgs_sweeps(A: sp.csr_matrix, grid: Grid, g, lo, hi, sweeps, s=None):
    """Symmetric multicolour projected Gauss-Seidel for min g.s + 1/2 s.As,
    lo <= s <= hi (Sec. 4.2.2; the colouring is the parallel form of
    Gauss-Seidel the paper names for GPUs).  One sweep: colours
    0 .. 2^d-1 with the fields of a node in order 0 .. d, then colours
    2^d-1 .. 0 with fields d .. 0; each dof i takes
    s_i <- clamp(s_i - (g + A s)_i / A_ii, lo_i, hi_i) (skipped where
    A_ii <= 0), with the latest values of all others."""
    d, N = grid.dim, grid.N
    F = d + 1
    s = np.zeros_like(g) if s is None else s.copy()
    diag = A.diagonal()
    col = node_parity_colours(grid)
    order = [(c, f) for c in range(1 << d) for f in range(F)]
    for _ in range(sweeps):
        for c, f in order + order[::-1]:
            idx = f * N + np.where(col == c)[0]
            r = g[idx] + A[idx] @ s
            dd = diag[idx]
            pos = dd > 0.0
            new = s[idx].copy()
            new[pos] = np.minimum(np.maximum(s[idx][pos] - r[pos] / dd[pos], lo[idx][pos]), hi[idx][pos])
            s[idx] = new
    return s


QP_CG = 0
QP_PAPER = 1


def mprgp(Hv, g, lo, hi, dscale, tol, maxit, gamma=1.0, lam_max=None):
    """MPRGP (Dostal's modified proportioning with reduced gradient
    projections) for min g.s + 1/2 s.Hs, lo <= s <= hi, on the diagonally
    scaled problem y = D^(1/2) s (D = dscale, the positive diagonal; 1 where
    it is not): A = D^(-1/2) H D^(-1/2), b = -D^(-1/2) g.  Steps:
    - proportional iterate (||beta||^2 <= gamma^2 phi~.phi): a CG step on
      the free set if it stays feasible, else an expansion step (the
      feasible part of it, then a projected gradient step of length abar on
      the free gradient) and a CG restart;
    - otherwise a proportioning step along the chopped gradient beta.
    Stops when ||phi + beta|| <= tol (tol None: the forcing tolerance
    min(0.1, sqrt(|nu0|)) |nu0| of the first projected gradient nu0) or
    after maxit products.  abar = 1 / lam_max (lam_max: an upper estimate of
    ||A||).  Returns s."""
    sq = np.sqrt(dscale)
    A = lambda y: Hv(y / sq) / sq
    b = -g / sq
    l, u = lo * sq, hi * sq
    y = np.minimum(np.maximum(np.zeros_like(g), l), u)
    abar = 1.0 / lam_max

    def split(y, gr):
        # free: strictly inside; chopped: on a bound of a dof that can move
        # (l < u), pointing out of the box; fixed dofs (l = u) count in neither
        free = (l < y) & (y < u)
        movable = l < u
        beta = np.where(~free & movable & (y <= l), np.minimum(gr, 0.0), 0.0) + \
            np.where(~free & movable & (y >= u), np.maximum(gr, 0.0), 0.0)
        phi = np.where(free, gr, 0.0)
        # reduced free gradient for the proportionality test
        pt = np.where(phi > 0, np.minimum((y - l) / abar, phi), np.maximum((y - u) / abar, phi))
        pt = np.where(free, pt, 0.0)
        return free, phi, beta, pt

    gr = A(y) - b
    used = 1
    free, phi, beta, pt = split(y, gr)
    p = phi.copy()
    if tol is None:
        nu0 = float(np.linalg.norm(phi + beta))
        tol = min(0.1, math.sqrt(nu0)) * nu0
    while used < maxit and np.linalg.norm(phi + beta) > tol:
        if float(beta @ beta) <= gamma * gamma * float(pt @ phi):
            Ap = A(p)
            used += 1
            pAp = float(p @ Ap)
            if pAp <= 0.0:
                break
            acg = float(gr @ p) / pAp
            # largest feasible step along -p
            with np.errstate(divide="ignore", invalid="ignore"):
                af = np.min(np.where(p > 0, (y - l) / p, np.where(p < 0, (y - u) / p, np.inf)))
            if acg <= af:
                y = y - acg * p
                gr = gr - acg * Ap
                free, phi, beta, pt = split(y, gr)
                gam = float(phi @ Ap) / pAp
                p = phi - gam * p
            else:
                y = y - af * p
                gr = gr - af * Ap
                free, phi, _, _ = split(y, gr)
                y = np.minimum(np.maximum(y - abar * phi, l), u)
                gr = A(y) - b
                used += 1
                free, phi, beta, pt = split(y, gr)
                p = phi.copy()
        else:
            d = beta
            Ad = A(d)
            used += 1
            dAd = float(d @ Ad)
            if dAd <= 0.0:
                break
            a = float(gr @ d) / dAd
            y = y - a * d
            gr = gr - a * Ad
            free, phi, beta, pt = split(y, gr)
            p = phi.copy()
    return y / sq


def paper_subproblem(model, g, lo, hi, tr: TRParams, stats=None):
    """The TR subproblem eq. (model_qp) with the paper's QP solvers
    (Sec. 4.2.2): MPRGP on the coarsest level (cg_coarse products, forcing
    tolerance, expansion step from the Gershgorin bound of the diagonally
    scaled Hessian), tr.pgs_sweeps symmetric PGS sweeps from s = 0 on the
    other levels.  The level's lagged model Hessian is taken as a sparse
    matrix by probing, once per lag."""
    if not hasattr(model, "_sparse"):
        model._sparse = probe_sparse(model.H.grids[model.level], model.Hlag)
    A = model._sparse
    if model.level == 0:
        dd = A.diagonal()
        dd = np.where(dd > 0.0, dd, 1.0)
        sq = np.sqrt(dd)
        lam = float(np.max(np.asarray(abs(sp.diags(1 / sq) @ A @ sp.diags(1 / sq)).sum(axis=1)).ravel()))
        return mprgp(lambda v: A @ v, g, lo, hi, dd, None, tr.cg_coarse, lam_max=lam)
    return pgs_sweeps(A, model.H.grids[model.level], g, lo, hi, tr.pgs_sweeps)


# --------------------------------------------------------------------------
# levels and the level objective h^l (eq. second_order_consistency)
# --------------------------------------------------------------------------
class Hierarchy:
    def __init__(self, dim, n_coarse, h_coarse, n_levels, prm: Params, ls_over_h=2.0):
        self.dim = dim
        self.L = n_levels
        self.grids = []
        for l, n in enumerate(level_sizes(n_coarse, n_levels)):
            self.grids.append(Grid(dim, n, h_coarse / 2 ** l))
        self.fine = self.grids[-1]
        self.prm = prm
        self.prm.ls = ls_over_h * self.fine.h  # l_s = 2 h on every level (Sec. 5)
        self.transfers = [Transfer(self.grids[l], self.grids[l + 1]) for l in range(n_levels - 1)]
        self.c_prev = np.zeros(self.fine.N)

    def ndof(self, level):
        return (self.dim + 1) * self.grids[level].N

    def dirichlet_mask(self, level):
        """True on displacement dofs of boundary nodes (clamped, u = 0)."""
        g = self.grids[level]
        bnd = g.boundary_nodes()
        m = np.zeros((self.dim + 1) * g.N, dtype=bool)
        for i in range(self.dim):
            m[i * g.N:(i + 1) * g.N] = bnd
        return m

    def fine_bounds(self):
        """Feasible set F of eq. (space_pf): c_prev <= c <= 1, u free except
        the clamped boundary."""
        g = self.fine
        d, N = self.dim, g.N
        lb = np.full((d + 1) * N, -np.inf)
        ub = np.full((d + 1) * N, np.inf)
        lb[d * N:] = self.c_prev
        ub[d * N:] = 1.0
        m = self.dirichlet_mask(self.L - 1)
        lb[m] = 0.0
        ub[m] = 0.0
        return lb, ub

    def f(self, level, x):
        return energy(self.grids[level], self.prm, x)

    def df(self, level, x):
        return gradient(self.grids[level], self.prm, x)

    def d2f(self, level, x, v):
        return hessvec(self.grids[level], self.prm, x, v)


class LevelModel:
    """h^l of eq. (second_order_consistency) at one level of one V-cycle.

    Finest level: h = f, model Hessian = Hessian of f at the lagged point.
    Coarser level: h(x) = f~(x) + <dg, x - x0> + 1/2 <x - x0, dH (x - x0)>
    with dg, dH from eq. (delta_terms); under Hessian lagging the model
    Hessian is R H_{l+1} I (GALERKIN) or Hess f~(x0) (FIRST_ORDER)."""

    def __init__(self, H: Hierarchy, level, x_lag, finer=None, dg=None, kind=FIRST_ORDER):
        self.H, self.level, self.kind = H, level, kind
        self.x_lag = x_lag.copy()
        self.finer = finer
        self.dg = dg
        self.x0 = x_lag.copy()
        self.stats = None

    @property
    def finest(self):
        return self.finer is None

    def Hlag(self, v):
        """Lagged model Hessian applied to v."""
        if self.finest or self.kind == FIRST_ORDER:
            return self.H.d2f(self.level, self.x_lag, v)
        T = self.H.transfers[self.level]
        return T.restrict(self.finer.Hlag(T.prolong(v)))

    def minv(self):
        """Inverse of the positive part of a Hessian diagonal (Jacobi): the
        lagged Hessian's own diagonal on the finest level and for
        FIRST_ORDER; the diagonal of Hess f~(x0) for GALERKIN levels."""
        if not hasattr(self, "_minv"):
            grid = self.H.grids[self.level]
            dd = hess_diag(grid, self.H.prm, self.x_lag)
            self._minv = np.where(dd > 0.0, 1.0 / np.where(dd > 0.0, dd, 1.0), 0.0)
        return self._minv

    def dH(self, v):
        if self.finest or self.kind == FIRST_ORDER:
            return np.zeros_like(v)
        return self.Hlag(v) - self.H.d2f(self.level, self.x0, v)

    def value(self, x):
        if self.finest:
            return self.H.f(self.level, x)
        s = x - self.x0
        return self.H.f(self.level, x) + float(self.dg @ s) + 0.5 * float(s @ self.dH(s))

    def diff(self, x, s):
        """h(x + s) - h(x), evaluated without subtracting two totals."""
        fd = energy_diff(self.H.grids[self.level], self.H.prm, x, s)
        if self.finest:
            return fd
        return fd + float(self.dg @ s) + float(s @ self.dH(x - self.x0)) + 0.5 * float(s @ self.dH(s))

    def grad(self, x):
        if self.finest:
            return self.H.df(self.level, x)
        s = x - self.x0
        return self.H.df(self.level, x) + self.dg + self.dH(s)


def convergence_control(rho, x, s, delta, lb, ub, tr: TRParams):
    """Algorithm 3: accept if rho > eta1; radius update gamma1/keep/gamma2.
    The accepted iterate is clipped to the bounds so that it stays feasible
    bit for bit."""
    if rho > tr.eta1:
        x = np.minimum(np.maximum(x + s, lb), ub)
    if rho < tr.eta1:
        delta = tr.gamma1 * delta
    elif rho > tr.eta2:
        delta = min(tr.gamma2 * delta, tr.delta_max)
    return x, delta


def nonlinear_solve(model: LevelModel, x0, lb, ub, delta0, iters, cg_max, tr: TRParams, stats):
    """Algorithm 2: `iters` trust-region iterations on h with the lagged
    model Hessian, each solving eq. (model_qp) and testing eq. (rho_tr).
    A non-finest level also stops once its projected gradient has fallen
    by level_rtol (when level_rtol > 0)."""
    x = x0.copy()
    delta = delta0
    minv = model.minv() if tr.precondition else None
    chi0 = None
    for _ in range(iters):
        g = model.grad(x)
        if tr.level_rtol > 0.0 and not model.finest:
            chi = projected_gradient_norm(x, g, lb, ub)
            if chi0 is None:
                chi0 = chi
            elif chi <= tr.level_rtol * chi0:
                break
        lo = np.maximum(lb - x, -delta)
        hi = np.minimum(ub - x, delta)
        if tr.qp_solver == QP_PAPER:
            s = paper_subproblem(model, g, lo, hi, tr, stats)
        else:
            s = solve_subproblem(g, model.Hlag, lo, hi, delta, cg_max, tr, stats, minv)
        pred = -(float(g @ s) + 0.5 * float(s @ model.Hlag(s)))
        stats["hessvecs"] += 1
        stats["tr_its"] += 1
        lv = stats.setdefault("tr_level", {})
        lv[model.level] = lv.get(model.level, 0) + 1
        if not pred > 0.0:
            break
        rho = -model.diff(x, s) / pred
        if rho <= tr.eta1:
            stats["tr_rejected"] += 1
            rj = stats.setdefault("rej_level", {})
            rj[model.level] = rj.get(model.level, 0) + 1
        x, delta = convergence_control(rho, x, s, delta, lb, ub, tr)
    return x, delta


def vcycle(H: Hierarchy, level, model: LevelModel, x0, lb, ub, delta0, tr: TRParams, stats):
    """Algorithm 1 (V-cycle of RMTR) with mu1 = mu2 = 1 and Hessian lagging."""
    cg = tr.cg_fine if model.finest else tr.cg_smooth
    x, delta = nonlinear_solve(model, x0, lb, ub, delta0, tr.mu1, cg, tr, stats)
    if level == 0:
        return x, delta
    T = H.transfers[level - 1]
    # coarse feasible set F^{l-1}: bounds of the fine correction at x_mu1
    lo_f = np.maximum(lb - x, -delta)
    hi_f = np.minimum(ub - x, delta)
    lo_c = T.support_max(lo_f)
    hi_c = T.support_min(hi_f)
    x0c = T.project(x)
    lbc = x0c + lo_c
    ubc = x0c + hi_c
    # coarse objective: dg = R grad h^l(x_mu1) - grad f~(x0c)
    Rg = T.restrict(model.grad(x))
    dg = Rg - H.df(level - 1, x0c)
    coarse = LevelModel(H, level - 1, x0c, finer=model, dg=dg, kind=tr.coarse_model)
    # the finer model's lag point stays fixed (Hessian lagging)
    if level - 1 == 0:
        xc, _ = nonlinear_solve(coarse, x0c, lbc, ubc, delta, tr.coarse_its, tr.cg_coarse, tr, stats)
    else:
        xc, _ = vcycle(H, level - 1, coarse, x0c, lbc, ubc, delta, tr, stats)
    s = T.prolong(xc - x0c)
    pred = -coarse.diff(x0c, xc - x0c)
    if pred > 0.0:
        rho = -model.diff(x, s) / pred
        if rho <= tr.eta1:
            stats["coarse_rejected"] += 1
        x, delta = convergence_control(rho, x, s, delta, lb, ub, tr)
    x, delta = nonlinear_solve(model, x, lb, ub, delta, tr.mu2, cg, tr, stats)
    return x, delta


def trust_region_gate(H: Hierarchy, x, xhat, eta):
    """Acceptance of a proposed iterate xhat at the current pressure by the
    trust-region ratio of eq. (rho_tr) and Algorithm 3's acceptance test
    (rho > eta1), as the learned initial iterate uses it (the paper has no
    learned part; the ratio and the test are the paper's):
    c_prev := c of x; s = P_F(xhat) - x with F the feasible set of
    eq. (space_pf) (c_prev <= c <= 1, clamped u); actual = E(x) - E(x + s),
    evaluated as the exact quartic expansion along s like every ratio here
    (the plain difference of two energies of size 1 loses the digits of a
    reduction of size 1e-7); predicted = -(grad E(x).s + s.H(x)s / 2);
    rho = actual / predicted
    (-inf when predicted <= 0); accepted when rho > eta and actual > 0.
    Returns (rho, accepted, the new x)."""
    d, N = H.dim, H.fine.N
    H.c_prev = x[d * N:].copy()
    lb, ub = H.fine_bounds()
    s = np.minimum(np.maximum(xhat, lb), ub) - x
    g = H.fine
    actual = -energy_diff(g, H.prm, x, s)
    pred = -(float(gradient(g, H.prm, x) @ s) + 0.5 * float(s @ hessvec(g, H.prm, x, s)))
    rho = actual / pred if pred > 0.0 else -math.inf
    acc = bool(rho > eta and actual > 0.0)
    return rho, acc, (x + s if acc else x.copy())


def projected_gradient_norm(x, g, lb, ub) -> float:
    """|| x - proj_F(x - grad f(x)) ||_2, the first-order criticality measure."""
    return float(np.linalg.norm(x - np.minimum(np.maximum(x - g, lb), ub)))


@dataclass
class LoadStepResult:
    x: np.ndarray
    cycles: int
    converged: bool
    energy: float
    pg0: float
    pg: float
    stats: dict = field(default_factory=dict)


def rmtr_load_step(H: Hierarchy, x, tr: TRParams = None, p=None) -> LoadStepResult:
    """One pseudo-time step: c_prev <- c, then RMTR V-cycles until the
    projected gradient has dropped by rtol (or max_cycles)."""
    tr = tr or TRParams()
    if p is not None:
        H.prm.p = p
    g0 = H.fine
    d, N = H.dim, g0.N
    x = x.copy()
    H.c_prev = x[d * N:].copy()
    lb, ub = H.fine_bounds()
    x = np.minimum(np.maximum(x, lb), ub)
    stats = dict(hessvecs=0, cg=0, tr_its=0, tr_rejected=0, coarse_rejected=0)
    pg0 = projected_gradient_norm(x, H.df(H.L - 1, x), lb, ub)
    pg = pg0
    delta = tr.delta0
    cycles = 0
    ref = tr.pg_ref if tr.pg_ref > 0 else pg0
    target = max(tr.rtol * ref, tr.atol)
    converged = pg0 <= (target if tr.pg_ref > 0 else tr.atol)
    while not converged and cycles < tr.max_cycles:
        model = LevelModel(H, H.L - 1, x)
        x, delta = vcycle(H, H.L - 1, model, x, lb, ub, delta, tr, stats)
        cycles += 1
        pg = projected_gradient_norm(x, H.df(H.L - 1, x), lb, ub)
        converged = pg <= target
    return LoadStepResult(x, cycles, converged, H.f(H.L - 1, x), pg0, pg, stats)
