"""FP64 CPU oracle for diag(H(i w_k)^-1): the exact diagonal and the paper's
Lanczos-based low-rank correction method (Carrier, Tang, Saad, Freericks,
"Lanczos-based Low-Rank Correction Method for Solving the Dyson Equation in
Inhomogeneous Dynamical Mean-Field Theory").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this module: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
leg use it.  It shares no code with the CUDA path; inputs come in as plain
numpy arrays.

Everything is complex128 / float64.  Library primitives used as single steps:
numpy matmul and numpy.linalg.inv for small dense blocks, numpy sqrt for the
principal complex square root.  There is no blocking, fusion or reordering
beyond what the paper's formulas state.

Site order: natural, x fastest, i = x + Lx*(y + Ly*z).

Readings of the paper taken here (the paper is silent or garbled there):
  * H = z I + t A with A the nearest-neighbour adjacency and
    z_i = i w + mu - V_i - Sigma_i(i w)                       (Eq. 1, Sec. 1 text)
  * domain decomposition: the slowest axis is cut into p strips (2D) or
    slabs (3D) separated by single interface lines/planes; the first
    (L_slow - p + 1) mod p strips get one extra layer        (Sec. 2.2, Fig. 1)
  * the start vector q1 is a caller-supplied real vector, normalised in the
    bilinear form                                             (Sec. 2.3)
  * diag(Q T Q^T) = sum_j alpha_j q_j*q_j + 2 sum_{j>=2} beta_j q_{j-1}*q_j
    with T = tridiag(beta_j, alpha_j, beta_{j+1})             (Eq. 9 text)
  * stop when ||r||_2 <= 1e-12 max|T| (the new residual vanished: invariant
    subspace reached; the paper names the 2-norm test as an alternative
    stopping rule); breakdown when r does not vanish but its bilinear "norm"
    does, |r^T r| <= 1e-14 ||r||_2^2 (Sec. 2.1, 2.3).  The 2-norm test comes
    first, so an exactly vanishing (r, r)_C with r != 0 is a breakdown and not
    a termination.
  * the H solve of Eq. 6 is a direct block-LU solve of the full lattice
    (the paper does not say which solver it used).
  * recursive decomposition (Sec. 2.3 end; 2D): a box is cut in two by one
    interface line through its middle, the cut direction alternating level by
    level; boxes of at most min_sites sites are inverted directly.
  * block Lanczos (not in the paper; for degenerate spectra of X): blocks are
    split by a column-by-column bilinear Gram-Schmidt QR (applied twice);
    a column whose 2-norm falls to 1e-12 max|T| is deflated to zero; the run
    terminates when a whole new block deflates; k_max counts columns.
"""
from __future__ import annotations

import numpy as np

STATUS_OK = 0
STATUS_TERMINATED = 1      # invariant subspace reached before the rank cap
STATUS_BREAKDOWN = 2       # (r, r)_C vanished for a non-zero r

# --------------------------------------------------------------------------
# Lattice and the Dyson matrix  (Eq. 1 and the text that follows it)
# --------------------------------------------------------------------------


def site_count(L) -> int:
    return int(np.prod(L))


def dyson_diagonal(omega: float, mu: float, V: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """H_ii(i w) = i w + mu - V_i - Sigma_i(i w)   (Eq. 1; Sec. 1, the noninteracting inverse)."""
    return 1j * omega + mu - V - sigma


def dyson_diagonal_real(omega: float, eta: float, mu: float, V: np.ndarray,
                        sigma: np.ndarray) -> np.ndarray:
    """Real-frequency form of Eq. 1, i w -> w + i eta (the remark after Eq. 1):
    H_ii(w) = w + i eta + mu - V_i - Sigma_i(w), Sigma the retarded self-energy."""
    return omega + 1j * eta + mu - V - sigma


def _axis_pairs(dims, periodic):
    """Nearest-neighbour pairs (i, j) of a box with dims (first fastest)."""
    n = int(np.prod(dims))
    idx = np.arange(n).reshape(tuple(reversed(dims)))      # idx[..., x]
    pairs = []
    nd = len(dims)
    for a in range(nd):
        ax = nd - 1 - a                                     # numpy axis of dim a
        lo = np.take(idx, np.arange(dims[a] - 1), axis=ax).ravel()
        hi = np.take(idx, np.arange(1, dims[a]), axis=ax).ravel()
        pairs.append(np.stack([lo, hi], 1))
        if periodic[a]:
            if dims[a] < 3:
                raise ValueError("periodic axes need at least 3 sites")
            lo = np.take(idx, [dims[a] - 1], axis=ax).ravel()
            hi = np.take(idx, [0], axis=ax).ravel()
            pairs.append(np.stack([lo, hi], 1))
    return np.concatenate(pairs, 0) if pairs else np.zeros((0, 2), dtype=int)


def adjacency(dims, periodic) -> np.ndarray:
    """Dense 0/1 nearest-neighbour adjacency of a box (first dim fastest)."""
    n = int(np.prod(dims))
    A = np.zeros((n, n))
    for i, j in _axis_pairs(list(dims), list(periodic)):
        A[i, j] = 1.0
        A[j, i] = 1.0
    return A


def dense_H(L, periodic, t: float, z: np.ndarray) -> np.ndarray:
    """H_ij = t_ij + z_i delta_ij with t_ij = t on nearest neighbours (Eq. 1)."""
    return np.diag(z).astype(np.complex128) + t * adjacency(L, periodic)


# --------------------------------------------------------------------------
# Dense inverse by LU with partial pivoting (the LAPACK route of Sec. 3,
# written out) -- for small N only.
# --------------------------------------------------------------------------


def lu_factor(Ain: np.ndarray):
    """Doolittle LU with row partial pivoting: P A = L U, stored in one array."""
    A = np.array(Ain, dtype=np.complex128, copy=True)
    n = A.shape[0]
    perm = np.arange(n)
    for k in range(n):
        piv = k + int(np.argmax(np.abs(A[k:, k])))
        if piv != k:
            A[[k, piv]] = A[[piv, k]]
            perm[[k, piv]] = perm[[piv, k]]
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, perm


def lu_inverse(Ain: np.ndarray) -> np.ndarray:
    """G = U^-1 L^-1 P: solve L U X = P I column block by forward/back substitution."""
    LU, perm = lu_factor(Ain)
    n = LU.shape[0]
    X = np.eye(n, dtype=np.complex128)[perm]
    for i in range(n):                      # forward: unit lower triangle
        X[i] -= LU[i, :i] @ X[:i]
    for i in range(n - 1, -1, -1):          # backward: upper triangle
        X[i] = (X[i] - LU[i, i + 1:] @ X[i + 1:]) / LU[i, i]
    return X


def dense_diag_inverse(L, periodic, t, z) -> np.ndarray:
    """diag(H^-1) from the dense LU inverse (Sec. 3, the original LAPACK route)."""
    return np.diag(lu_inverse(dense_H(L, periodic, t, z))).copy()


# --------------------------------------------------------------------------
# Block-tridiagonal structure along x: slice s = all sites with x = s.
# Within a slice the local index is j = y + Ly*z, so site = s + Lx*j.
# Consecutive slices couple through t*I.
# --------------------------------------------------------------------------


def slice_blocks(Lx: int, trans_dims, periodic_trans, t: float, z_slices):
    """D_s = diag(z on slice s) + t * (in-slice adjacency), s = 0..Lx-1."""
    A = adjacency(trans_dims, periodic_trans)
    return [np.diag(z_slices[s]).astype(np.complex128) + t * A for s in range(Lx)]


def block_tridiag_factor(D, t: float):
    """Left-connected inverses g_s = (D_s - t^2 g_{s-1})^-1 and diag(G_ss).

    Backward pass G_ss = g_s + t^2 g_s G_{s+1,s+1} g_s (the recursion that
    gives the diagonal blocks of a block-tridiagonal inverse; used for the
    exact diagonal and for diag(B^-1), Sec. 2.3 after Eq. 8).
    """
    g = []
    prev = None
    for Ds in D:
        A = Ds if prev is None else Ds - (t * t) * prev
        prev = np.linalg.inv(A)
        g.append(prev)
    n = len(D)
    diags = [None] * n
    G = g[-1]
    diags[-1] = np.diag(G).copy()
    for s in range(n - 2, -1, -1):
        G = g[s] + (t * t) * (g[s] @ G @ g[s])
        diags[s] = np.diag(G).copy()
    return g, diags


def block_tridiag_solve(g, t: float, rhs):
    """Block forward/back substitution with the stored g_s (rhs: list of slice vectors)."""
    n = len(g)
    y = [None] * n
    prev = None
    for s in range(n):
        zs = rhs[s] if prev is None else rhs[s] - t * prev
        prev = g[s] @ zs
        y[s] = prev
    x = [None] * n
    x[-1] = y[-1]
    for s in range(n - 2, -1, -1):
        x[s] = y[s] - t * (g[s] @ x[s + 1])
    return x


def _check_x_open(periodic):
    if periodic[0]:
        raise ValueError("the slice recursion runs along x, which must be open")


def exact_diag(L, periodic, t, z) -> np.ndarray:
    """Exact diag(H^-1) by the full-lattice block-tridiagonal recursion along x."""
    _check_x_open(periodic)
    Lx = L[0]
    trans = list(L[1:])
    zz = np.asarray(z).reshape(-1, Lx)            # zz[j, x]
    D = slice_blocks(Lx, trans, periodic[1:len(L)], t, [zz[:, s] for s in range(Lx)])
    _, diags = block_tridiag_factor(D, t)
    out = np.empty((zz.shape[0], Lx), dtype=np.complex128)
    for s in range(Lx):
        out[:, s] = diags[s]
    return out.ravel()


# --------------------------------------------------------------------------
# Domain decomposition ordering (Sec. 2.2, Fig. 1; Eq. 3)
# --------------------------------------------------------------------------


def dd_partition(L, p: int):
    """Split the slowest axis into p subdomains separated by p-1 single layers.

    Returns (starts, heights, interface_layers): subdomain i covers slow
    coordinates [starts[i], starts[i] + heights[i]); interface layer l sits
    at slow coordinate interface_layers[l] between subdomains l and l+1.
    The first (L_slow - p + 1) mod p subdomains get one extra layer.
    """
    Ls = L[-1]
    if p < 1 or Ls - (p - 1) < p:
        raise ValueError("too many subdomains for this lattice")
    base, extra = divmod(Ls - (p - 1), p)
    heights = [base + (1 if i < extra else 0) for i in range(p)]
    starts, layers = [], []
    c = 0
    for i in range(p):
        starts.append(c)
        c += heights[i]
        if i < p - 1:
            layers.append(c)
            c += 1
    assert c == Ls
    return starts, heights, layers


def dd_sites(L, p: int):
    """Natural indices in domain-decomposition order (Fig. 1 right).

    Subdomain i lists its sites slice by slice (x = 0..Lx-1); inside a slice
    the order is tr + T*sl, tr the transverse coordinate (y in 3D, absent in
    2D, T = 1 then) and sl the slow coordinate relative to the subdomain
    start.  Interface layers follow, each in order x + Lx*tr.
    """
    Lx = L[0]
    T = 1 if len(L) == 2 else L[1]
    A = Lx * T
    starts, heights, layers = dd_partition(L, p)
    sub = []
    for i in range(p):
        s0, h = starts[i], heights[i]
        idx = np.empty((Lx, T * h), dtype=np.int64)
        for x in range(Lx):
            for sl in range(h):
                for tr in range(T):
                    idx[x, tr + T * sl] = x + Lx * tr + A * (s0 + sl)
        sub.append(idx)
    iface = [np.array([x + Lx * tr + A * yl for tr in range(T) for x in range(Lx)],
                      dtype=np.int64) for yl in layers]
    return sub, iface


class Subdomains:
    """The B blocks of Eq. 3: per-subdomain slice factors g_s and diag(B^-1)."""

    def __init__(self, L, periodic, t, z, p):
        _check_x_open(periodic)
        if len(L) == 3 and periodic[2] and p > 1:
            raise ValueError("the split axis must be open")
        if len(L) == 2 and periodic[1] and p > 1:
            raise ValueError("the split axis must be open")
        self.L, self.t, self.p = L, t, p
        self.sub, self.iface = dd_sites(L, p)
        _, heights, _ = dd_partition(L, p)
        Lx = L[0]
        trans_p = [periodic[1]] if len(L) == 3 else []
        slow_p = periodic[len(L) - 1] if p == 1 else False
        self.g = []
        self.diagB = np.zeros(site_count(L), dtype=np.complex128)
        for i, idx in enumerate(self.sub):
            dims = ([L[1]] if len(L) == 3 else []) + [heights[i]]
            D = slice_blocks(Lx, dims, trans_p + [slow_p], t, [z[idx[s]] for s in range(Lx)])
            g, diags = block_tridiag_factor(D, t)
            self.g.append(g)
            for s in range(Lx):
                self.diagB[idx[s]] = diags[s]

    def solve(self, q: np.ndarray) -> np.ndarray:
        """w = blkdiag(B^-1, 0) q   (Eq. 7): subdomain solves, zero on the interface."""
        w = np.zeros_like(q, dtype=np.complex128)
        for g, idx in zip(self.g, self.sub):
            x = block_tridiag_solve(g, self.t, [q[idx[s]] for s in range(idx.shape[0])])
            for s in range(idx.shape[0]):
                w[idx[s]] = x[s]
        return w


class FullLattice:
    """Direct solver for H v = q (Eq. 6) by block LU along x of the whole lattice."""

    def __init__(self, L, periodic, t, z):
        _check_x_open(periodic)
        self.L, self.t = L, t
        Lx = L[0]
        zz = np.asarray(z).reshape(-1, Lx)
        D = slice_blocks(Lx, list(L[1:]), periodic[1:len(L)], t, [zz[:, s] for s in range(Lx)])
        self.g, _ = block_tridiag_factor(D, t)

    def solve(self, q: np.ndarray) -> np.ndarray:
        Lx = self.L[0]
        qq = np.asarray(q, dtype=np.complex128).reshape(-1, Lx)
        x = block_tridiag_solve(self.g, self.t, [qq[:, s] for s in range(Lx)])
        return np.stack(x, 1).ravel()


# --------------------------------------------------------------------------
# Complex-symmetric Lanczos in the bilinear form (Sec. 2.1 after Freund et al.;
# Sec. 2.3 Eqs. 5, 9 and the stopping discussion)
# --------------------------------------------------------------------------


def cs_lanczos(matvec, q1, k_max: int, term_tol: float = 1e-12, brk_tol: float = 1e-14,
               branch: int = 1):
    """Lanczos on a complex-symmetric operator with (q, u)_C = q^T u.

    Full re-orthogonalisation, classical Gram-Schmidt applied twice, in the
    same bilinear form.  Accumulates diag(Q_k T_k Q_k^T) with the three-vector
    update of Sec. 2.3 while the recurrence runs.

    Returns (diag_QTQ, alphas, betas, Q, status) where betas[j] couples
    q_{j+1} and q_{j+2} (0-based Q columns j and j+1).  branch = -1 takes the
    other square root for every beta (the result must not change).
    """
    q1 = np.asarray(q1, dtype=np.complex128)
    N = q1.shape[0]
    acc = np.zeros(N, dtype=np.complex128)
    alphas, betas = [], []
    if k_max <= 0:
        return acc, np.array(alphas), np.array(betas), np.zeros((N, 0), complex), STATUS_OK
    Q = np.zeros((N, k_max + 1), dtype=np.complex128)
    Q[:, 0] = q1 / np.sqrt(q1 @ q1)
    beta_prev = 0.0
    status = STATUS_OK
    for j in range(k_max):
        qj = Q[:, j]
        u = matvec(qj)
        a = qj @ u
        r = u - a * qj
        if j > 0:
            r = r - beta_prev * Q[:, j - 1]
        for _ in range(2):                       # CGS2 in the bilinear form
            h = Q[:, :j + 1].T @ r
            r = r - Q[:, :j + 1] @ h
        acc += a * qj * qj
        if j > 0:
            acc += 2.0 * beta_prev * Q[:, j - 1] * qj
        alphas.append(a)
        rr = r @ r
        rn2 = np.vdot(r, r).real                 # ||r||_2^2 (conjugated)
        b = branch * np.sqrt(rr)
        maxT = max(max(abs(x) for x in alphas), max((abs(x) for x in betas), default=0.0))
        if j == k_max - 1:
            break
        if np.sqrt(rn2) <= term_tol * maxT:      # r itself vanished: invariant subspace
            status = STATUS_TERMINATED
            break
        if abs(rr) <= brk_tol * rn2:             # r != 0 but (r, r)_C ~ 0: breakdown
            status = STATUS_BREAKDOWN
            break
        betas.append(b)
        Q[:, j + 1] = r / b
        beta_prev = b
    steps = len(alphas)
    return acc, np.array(alphas), np.array(betas), Q[:, :steps], status


def _bilinear_qr(R, maxT: float, term_tol: float, brk_tol: float):
    """R = Q B in the bilinear form, column by column (Gram-Schmidt twice).

    Q^T Q = I on the kept columns; a column whose 2-norm falls to
    term_tol * maxT is deflated (q_c = 0, B_cc = 0) and takes no further
    part.  Returns (Q, B, deflated[b], breakdown) where breakdown means
    (r, r)_C vanished for a column that is not small.
    """
    N, nb = R.shape
    Q = np.zeros((N, nb), dtype=np.complex128)
    B = np.zeros((nb, nb), dtype=np.complex128)
    defl = np.zeros(nb, dtype=bool)
    for c in range(nb):
        r = R[:, c].copy()
        for _ in range(2):
            h = Q[:, :c].T @ r
            r = r - Q[:, :c] @ h
            B[:c, c] += h
        rr = r @ r
        rn2 = np.vdot(r, r).real
        b = np.sqrt(rr)
        if np.sqrt(rn2) <= term_tol * maxT:      # the column vanished: deflate it
            defl[c] = True
            continue
        if abs(rr) <= brk_tol * rn2:             # r != 0 but (r, r)_C ~ 0: breakdown
            return Q, B, defl, True
        B[c, c] = b
        Q[:, c] = r / b
    return Q, B, defl, False


def cs_block_lanczos(matvec, Q1, k_max: int, term_tol: float = 1e-12, brk_tol: float = 1e-14):
    """Block complex-symmetric Lanczos with (q, u)_C = q^T u.

    Not in the paper: the block form of Sec. 2.1's recurrence, for X whose
    eigenvalues are degenerate (a single start vector spans only one
    direction of each eigenspace).  With block size nb = Q1.shape[1]:

        X Q_j = Q_{j-1} B_j^T + Q_j A_j + Q_{j+1} B_{j+1},
        A_j = Q_j^T X Q_j,   R_j = X Q_j - Q_j A_j - Q_{j-1} B_j^T = Q_{j+1} B_{j+1}

    with R_j re-orthogonalised against every earlier block (CGS2) and split
    by the bilinear QR above.  T is block tridiagonal (A_j on the diagonal,
    B_{j+1} below, B_{j+1}^T above), so the diagonal of Q T Q^T takes, per
    block step, diag(Q_j A_j Q_j^T) + 2 diag(Q_j B_j Q_{j-1}^T) (Eq. 9 per
    block).  k_max is the rank cap: k_max / nb block steps.  Stops when every
    column of the next block deflated (invariant subspace: terminated) or on a
    bilinear breakdown.  The start block is split by the same QR first.

    Returns (diag_QTQ, A[steps], B[steps], Q, status); B[j] couples block j
    to block j - 1 (B[0] = the start block's factor).
    """
    Q1 = np.asarray(Q1, dtype=np.complex128)
    N, nb = Q1.shape
    if k_max % nb:
        raise ValueError("k_max must be a multiple of the block size")
    nsteps = k_max // nb
    acc = np.zeros(N, dtype=np.complex128)
    Qj, B0, defl, brk = _bilinear_qr(Q1, 1.0, 0.0, brk_tol)
    if brk or defl.any():
        raise ValueError("start block is not of full rank in the bilinear form")
    blocks = [Qj]
    As, Bs = [], [B0]
    status = STATUS_OK
    maxT = 0.0
    for j in range(nsteps):
        Qj = blocks[j]
        U = matvec(Qj)
        A = Qj.T @ U
        Rj = U - Qj @ A
        if j > 0:
            Rj = Rj - blocks[j - 1] @ Bs[j].T
        Qall = np.concatenate(blocks, axis=1)
        for _ in range(2):                       # CGS2 in the bilinear form
            Rj = Rj - Qall @ (Qall.T @ Rj)
        acc += np.einsum("ic,cd,id->i", Qj, A, Qj)
        if j > 0:
            acc += 2.0 * np.einsum("ic,cd,id->i", Qj, Bs[j], blocks[j - 1])
        As.append(A)
        maxT = max(maxT, np.abs(A).max())
        if j == nsteps - 1:
            break
        Qn, Bn, defl, brk = _bilinear_qr(Rj, maxT, term_tol, brk_tol)
        if brk:
            status = STATUS_BREAKDOWN
            break
        if defl.all():
            status = STATUS_TERMINATED
            break
        maxT = max(maxT, np.abs(Bn).max())
        blocks.append(Qn)
        Bs.append(Bn)
    Q = np.concatenate(blocks[:len(As)], axis=1)
    return acc, np.array(As), np.array(Bs[:len(As)]), Q, status


# --------------------------------------------------------------------------
# The low-rank correction method (Sec. 2.3, Eqs. 4-9)
# --------------------------------------------------------------------------


def axis_diagonal(omega_k, mu, V, sigma_k, eta: float = 0.0) -> np.ndarray:
    """The Dyson diagonal on the Matsubara axis (eta = 0) or the real axis (eta > 0)."""
    if eta > 0.0:
        return dyson_diagonal_real(omega_k, eta, mu, V, sigma_k)
    return dyson_diagonal(omega_k, mu, V, sigma_k)


def lowrank_diag(L, periodic, t, mu, V, sigma_k, omega_k, q1, p: int, k_max: int,
                 return_info: bool = False, eta: float = 0.0):
    """diag(H^-1) = diag(blkdiag(B^-1, 0)) + diag(Q_k T_k Q_k^T)   (Eq. 9).

    X q = H^-1 q - blkdiag(B^-1, 0) q by one direct H solve and the
    subdomain solves (Eqs. 6-8); p = 1 has no interface, X = 0 and the
    result is the exact recursion.  eta > 0: real frequency axis.
    """
    z = axis_diagonal(omega_k, mu, V, sigma_k, eta)
    subs = Subdomains(L, periodic, t, z, p)
    if p == 1:
        acc = np.zeros(site_count(L), dtype=np.complex128)
        info = dict(alphas=np.zeros(0, complex), betas=np.zeros(0, complex), steps=0,
                    status=STATUS_OK, diagB=subs.diagB)
        return (subs.diagB + acc, info) if return_info else subs.diagB + acc
    full = FullLattice(L, periodic, t, z)

    def xmatvec(q):
        v = full.solve(q)          # Eq. 6
        w = subs.solve(q)          # Eq. 7
        return v - w               # Eq. 8

    acc, al, be, Q, status = cs_lanczos(xmatvec, q1, k_max)
    res = subs.diagB + acc
    if return_info:
        return res, dict(alphas=al, betas=be, steps=len(al), status=status,
                         diagB=subs.diagB, Q=Q)
    return res


def lowrank_diag_block(L, periodic, t, mu, V, sigma_k, omega_k, Q1, p: int, k_max: int,
                       return_info: bool = False, eta: float = 0.0):
    """Eq. 9 with the block Lanczos approximation of X (start block Q1, N x nb)."""
    z = axis_diagonal(omega_k, mu, V, sigma_k, eta)
    subs = Subdomains(L, periodic, t, z, p)
    full = FullLattice(L, periodic, t, z)

    def xmatvec_block(Qb):
        return np.stack([full.solve(Qb[:, c]) - subs.solve(Qb[:, c])
                         for c in range(Qb.shape[1])], axis=1)   # Eqs. 6-8 per column

    acc, As, Bs, Q, status = cs_block_lanczos(xmatvec_block, Q1, k_max)
    res = subs.diagB + acc
    if return_info:
        return res, dict(A=As, B=Bs, steps=len(As), status=status, diagB=subs.diagB, Q=Q)
    return res


def recursive_diag(L, t, z, q1, k_max: int, min_sites: int = 64, first_cut: str = "x", boxes=None):
    """diag(H^-1) by the recursive decomposition of Sec. 2.3 (end): 2D only.

    A box of the lattice (its principal submatrix of H, open at the box edges) is
    cut into two halves by one interface line, alternating the cut direction
    level by level, (d_x, d_y) = (2, 1), (1, 2), ... when first_cut = "x".  Its
    diagonal is [diag of each half's inverse, by the same method one level down;
    0 on the line] + diag(Q_k T_k Q_k^T) of X_box = H_box^-1 - blkdiag(H_1^-1,
    H_2^-1, 0) (Eqs. 5-9 applied to the box), with the start vector q1
    restricted to the box.  Boxes of at most min_sites sites are inverted
    directly.  With k_max past every level's closure the result is exact.
    Returns the diagonal in natural order.  If `boxes` is a list, every box
    visited is appended to it as (x0, y0, nx, ny, level, leaf, axis, line): the
    line is the column x = line (axis 0) or the row y = line (axis 1); axis and
    line are -1 for a leaf.
    """
    Lx, Ly = L
    z = np.asarray(z, dtype=np.complex128)
    q1 = np.asarray(q1, dtype=np.float64)

    def sites(x0, x1, y0, y1):
        return np.array([x + Lx * y for y in range(y0, y1 + 1) for x in range(x0, x1 + 1)], dtype=np.int64)

    def box_H(idx, nx, ny):
        return dense_H((nx, ny), (False, False), t, z[idx])

    def rec(x0, x1, y0, y1, cut, level=0):
        nx, ny = x1 - x0 + 1, y1 - y0 + 1
        idx = sites(x0, x1, y0, y1)
        Hb = box_H(idx, nx, ny)
        if idx.size <= min_sites or (cut == "x" and nx < 3) or (cut == "y" and ny < 3):
            if idx.size <= min_sites or (nx < 3 and ny < 3):
                if boxes is not None:
                    boxes.append((x0, y0, nx, ny, level, 1, -1, -1))
                return idx, np.diag(np.linalg.inv(Hb))
            cut = "y" if cut == "x" else "x"
        if cut == "x":
            xm = (x0 + x1) // 2
            halves = [(x0, xm - 1, y0, y1), (xm + 1, x1, y0, y1)]
        else:
            ym = (y0 + y1) // 2
            halves = [(x0, x1, y0, ym - 1), (x0, x1, ym + 1, y1)]
        if boxes is not None:
            boxes.append((x0, y0, nx, ny, level, 0, 0, xm) if cut == "x" else (x0, y0, nx, ny, level, 0, 1, ym))
        nxt = "y" if cut == "x" else "x"
        pos = {int(v): k for k, v in enumerate(idx)}
        parts = []
        for h in halves:
            hidx, hdiag = rec(*h, nxt, level + 1)
            parts.append((np.array([pos[int(v)] for v in hidx]), hidx, hdiag))
        d = np.zeros(idx.size, dtype=np.complex128)
        Hh = [box_H(hidx, h[1] - h[0] + 1, h[3] - h[2] + 1) for (_, hidx, _), h in zip(parts, halves)]

        def xmatvec(q):
            v = np.linalg.solve(Hb, q)                                  # Eq. 6 on the box
            w = np.zeros_like(v)
            for (loc, _, _), Hhalf in zip(parts, Hh):
                w[loc] = np.linalg.solve(Hhalf, q[loc])                 # Eq. 7: the halves
            return v - w                                                # Eq. 8

        acc = cs_lanczos(xmatvec, q1[idx].astype(np.complex128), k_max)[0]
        for loc, _, hdiag in parts:
            d[loc] = hdiag
        return idx, d + acc

    idx, d = rec(0, Lx - 1, 0, Ly - 1, first_cut)
    out = np.zeros(Lx * Ly, dtype=np.complex128)
    out[idx] = d
    return out


def xmatvec(L, periodic, t, mu, V, sigma_k, omega_k, p, q, eta: float = 0.0):
    """One X-'matvec' u = H^-1 q - blkdiag(B^-1, 0) q (Eqs. 6-8), natural order."""
    z = axis_diagonal(omega_k, mu, V, sigma_k, eta)
    subs = Subdomains(L, periodic, t, z, p)
    full = FullLattice(L, periodic, t, z)
    return full.solve(q) - subs.solve(q)


def xmatvec_cancel_free(L, periodic, t, mu, V, sigma_k, omega_k, p, q, eta: float = 0.0):
    """The same X q as xmatvec (Eqs. 6-8) through an equivalent form: with
    w = blkdiag(B^-1, 0) q, H (v - w) = q - H w, so u = H^-1 (q - H w).  The
    right-hand side vanishes on the subdomains up to rounding, so the
    subtraction of two nearly equal vectors in Eq. 8 is avoided.  Both forms
    give X q in exact arithmetic; their FP64 results differ at the rounding
    level, which measures how much FP64 rounding of the X-matvec moves the
    truncated Lanczos result."""
    z = axis_diagonal(omega_k, mu, V, sigma_k, eta)
    subs = Subdomains(L, periodic, t, z, p)
    full = FullLattice(L, periodic, t, z)
    w = subs.solve(q)
    return full.solve(q - apply_H(L, periodic, t, mu, V, sigma_k, omega_k, w, eta))


def apply_H(L, periodic, t, mu, V, sigma_k, omega_k, x, eta: float = 0.0):
    """y = H x by the stencil (Eq. 1), natural order, without forming H."""
    z = axis_diagonal(omega_k, mu, V, sigma_k, eta)
    y = z * x
    for i, j in _axis_pairs(list(L), list(periodic[:len(L)])):
        y[i] += t * x[j]
        y[j] += t * x[i]
    return y


# --------------------------------------------------------------------------
# Batched drivers over frequencies
# --------------------------------------------------------------------------


def exact_diag_batch(L, periodic, t, mu, V, sigma, omega):
    return np.stack([exact_diag(L, periodic, t, dyson_diagonal(w, mu, V, sigma[k]))
                     for k, w in enumerate(omega)])


def lowrank_diag_batch(L, periodic, t, mu, V, sigma, omega, q1, p, k_max):
    return np.stack([lowrank_diag(L, periodic, t, mu, V, sigma[k], w, q1, p, k_max)
                     for k, w in enumerate(omega)])


def subdomain_diag_batch(L, periodic, t, mu, V, sigma, omega, p):
    """diag(blkdiag(B^-1, 0)) per frequency (Eq. 9 first term), natural order."""
    return np.stack([Subdomains(L, periodic, t, dyson_diagonal(w, mu, V, sigma[k]), p).diagB
                     for k, w in enumerate(omega)])
