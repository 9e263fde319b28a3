"""Plain, slow, FP64 CPU oracle for exponential discriminant analysis (EDA).

TEST INFRASTRUCTURE ONLY (see the package docstring). Nothing here is tuned;
each function follows the paper's definitions in the paper's order. Library
primitives used as single steps: numpy matmul, ``numpy.linalg.eigh`` (a
symmetric eigendecomposition), ``numpy.linalg.qr`` (Householder QR),
``numpy.linalg.svd``, ``numpy.linalg.cholesky`` and ``numpy.linalg.eig`` (the
small Hessenberg matrix of the Arnoldi method).

Notation (Section 1, Table 1.1): X = [chi_1 .. chi_n] is d x n, k classes,
n_j samples in class j, mu_j class centroids, mu the global centroid, t the
number of wanted eigenpairs. Arrays here are natural d x n numpy matrices;
the ``X`` argument of the public functions is the (n, d) sample-per-row array
produced by ``paper_1512_06500_gb300.synth`` (the same memory as a
column-major d x n matrix).

Pins (what each function is checked against, in tests/test_oracle_*.py):
  segment ............ brute-force counting; stability by explicit loops
  scatter_factors .... exact rational means (fractions.Fraction); column sums
                       of H_W per class and sqrt(n_j)-weighted sum of H_B vanish
  jacobi_eigh ........ diagonal/2x2 closed forms; A U = U diag(w); U^T U = I
  expm_taylor ........ exp(0) = I; diagonal closed form; exp(A) exp(-A) = I;
                       agreement with the eigen route on random symmetric A
  sym_fun ............ same pins as expm_taylor through f = exp
  lowrank_exp_apply .. Theorem 3.1 identity against the dense Taylor route;
                       H = 0 gives Y = X exactly
  phi_operator ....... direct power series sum_j alpha^j G^(j-1) / j!
  eda_dense .......... commuting diagonal closed form; Example 1.1 closed
                       form; Theorem 3.3 bounds; Theorem 3.7 unit-eigenvalue
                       count; Cholesky route on d <= 8
  eda_projected ...... equality with eda_dense on d <= 256
  n_apply ............ the dense product exp(-c^2 S_W) exp(c^2 S_B) X
  eda_arnoldi ........ eigenvalues and eigenvector span of the symmetric route
                       (similarity N = E_W^{-1/2} M E_W^{1/2}); commuting
                       diagonal closed form; all d eigenvalues of the dense N
                       on d <= 12 (no GPU counterpart yet: the nonsymmetric
                       form is a next step of the library)
  nn_classify ........ brute force on tiny sets; Theorem 3.8 bound
None of the functions is "parity unpinned".
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "segment", "scatter_factors", "gram", "jacobi_eigh", "expm_taylor", "sym_fun",
    "lowrank_exp_apply", "dense_exp_apply", "phi", "phi_operator", "scale_c2",
    "m_apply", "eda_dense", "eda_projected", "eda", "project", "nn_classify",
    "sin_angle", "orth", "eda_cholesky_route", "trace_ratio", "n_apply", "eda_arnoldi",
]


# --------------------------------------------------------------------------
# Section 1: class partition, centroids and the scatter factors H_W, H_B
# --------------------------------------------------------------------------

def segment(labels, k):
    """Class partition of the samples (Section 1: X = [X_1, ..., X_k]).

    Returns (counts n_j, offsets, perm): perm lists the samples class by
    class (class 0 first) and, inside a class, in input order; offsets[j] is
    the position of class j's first sample in perm. Raises ValueError when a
    label is outside [0, k) or a class is empty (n_j >= 1 is assumed by the
    centroid definition).
    """
    labels = np.asarray(labels)
    n = labels.size
    counts = np.zeros(k, dtype=np.int64)
    for i in range(n):
        l = int(labels[i])
        if l < 0 or l >= k:
            raise ValueError(f"label {l} of sample {i} outside [0, {k})")
        counts[l] += 1
    if (counts == 0).any():
        raise ValueError(f"empty class {int(np.argmin(counts))}")
    offsets = np.zeros(k + 1, dtype=np.int64)
    for j in range(k):
        offsets[j + 1] = offsets[j] + counts[j]
    fill = offsets[:-1].copy()
    perm = np.empty(n, dtype=np.int64)
    for i in range(n):
        l = int(labels[i])
        perm[fill[l]] = i
        fill[l] += 1
    return counts.astype(np.int32), offsets.astype(np.int32), perm.astype(np.int32)


def scatter_factors(X, labels, k):
    """H_W (d x n) and H_B (d x k) of Eqs. (1.1) and (1.2).

    mu_j = (sum of the class-j samples, added one by one in input order) / n_j
    mu   = (sum of all samples, added one by one in input order) / n
    H_W[:, p] = chi_perm[p] - mu_{label}   (class-major columns, input order inside a class)
    H_B[:, j] = sqrt(n_j) * (mu_j - mu)
    Every step is a single IEEE double operation (no fused multiply-add), so the
    result is fixed bit for bit by this order.
    """
    X = np.asarray(X, dtype=np.float64)          # (n, d): row i = sample i
    n, d = X.shape
    counts, offsets, perm = segment(labels, k)
    mu_j = np.empty((k, d))
    for j in range(k):
        acc = np.zeros(d)
        for p in range(offsets[j], offsets[j + 1]):
            acc = acc + X[perm[p]]
        mu_j[j] = acc / np.float64(counts[j])
    acc = np.zeros(d)
    for i in range(n):
        acc = acc + X[i]
    mu = acc / np.float64(n)
    lab = np.asarray(labels)
    HW = np.empty((d, n))
    for p in range(n):
        i = perm[p]
        HW[:, p] = X[i] - mu_j[lab[i]]
    HB = np.empty((d, k))
    for j in range(k):
        HB[:, j] = np.sqrt(np.float64(counts[j])) * (mu_j[j] - mu)
    return dict(HW=HW, HB=HB, mu_j=mu_j, mu=mu, counts=counts, offsets=offsets, perm=perm)


def gram(H):
    """G = H^T H, the small Gram matrix whose spectrum is D = Sigma^2 of Eqs. (3.4)-(3.6)."""
    return H.T @ H


# --------------------------------------------------------------------------
# Section 2: the matrix exponential and functions of symmetric matrices
# --------------------------------------------------------------------------

def jacobi_eigh(A, tol=1e-15, max_sweeps=60):
    """Cyclic Jacobi eigendecomposition of a symmetric matrix (Golub and Van Loan, Section 8.5).

    Each rotation zeroes one off-diagonal pair; sweeps repeat until the
    off-diagonal Frobenius norm is below tol times the full norm.
    Returns (w ascending, U) with A = U diag(w) U^T.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    m = A.shape[0]
    U = np.eye(m)
    fro = np.linalg.norm(A)
    if fro == 0.0:
        return np.zeros(m), U
    for _ in range(max_sweeps):
        off = math.sqrt(np.sum(A * A * (1.0 - np.eye(m))))
        if off <= tol * fro:
            break
        for p in range(m - 1):
            for q in range(p + 1, m):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                theta = (A[q, q] - A[p, p]) / (2.0 * apq)
                tt = (1.0 if theta >= 0 else -1.0) / (abs(theta) + math.sqrt(1.0 + theta * theta))
                c = 1.0 / math.sqrt(1.0 + tt * tt)
                s = tt * c
                # A <- J^T A J with J the rotation in the (p, q) plane
                Ap = A[:, p].copy()
                Aq = A[:, q].copy()
                A[:, p] = c * Ap - s * Aq
                A[:, q] = s * Ap + c * Aq
                Ap = A[p, :].copy()
                Aq = A[q, :].copy()
                A[p, :] = c * Ap - s * Aq
                A[q, :] = s * Ap + c * Aq
                Up = U[:, p].copy()
                Uq = U[:, q].copy()
                U[:, p] = c * Up - s * Uq
                U[:, q] = s * Up + c * Uq
    w = np.diag(A).copy()
    order = np.argsort(w, kind="stable")
    return w[order], U[:, order]


def expm_taylor(A, degree=18):
    """exp(A) from its defining series (Section 2) by scaling and squaring.

    Pick j >= 0 with ||A||_1 / 2^j <= 1/2, sum the Taylor series of exp(A / 2^j)
    to the given degree by Horner's rule, then square j times.
    """
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    nrm = np.abs(A).sum(axis=0).max() if m else 0.0
    j = 0
    while nrm / (2.0 ** j) > 0.5:
        j += 1
    B = A / (2.0 ** j)
    E = np.eye(m)
    for i in range(degree, 0, -1):
        E = np.eye(m) + (B @ E) / i
    for _ in range(j):
        E = E @ E
    return E


def sym_fun(A, f, route="eigh"):
    """f(A) = U f(Lambda) U^T for symmetric A (Section 2: A and exp(A) share eigenvectors)."""
    A = 0.5 * (A + A.T)
    if route == "jacobi":
        w, U = jacobi_eigh(A)
    else:
        w, U = np.linalg.eigh(A)
    return (U * f(w)) @ U.T


def phi(z):
    """phi(z) = (e^z - 1) / z with phi(0) = 1, evaluated through expm1."""
    z = np.asarray(z, dtype=np.float64)
    out = np.ones_like(z)
    nz = z != 0.0
    out[nz] = np.expm1(z[nz]) / z[nz]
    return out


def phi_operator(G, alpha):
    """K(alpha) = alpha * phi(alpha G) for a symmetric PSD Gram G.

    With H = Q~ Sigma V^T (Eqs. (3.3)-(3.6)) and G = H^T H = V Sigma^2 V^T,
    Theorem 3.1 gives exp(alpha H H^T) = I + H K(alpha) H^T. Eigenvalues of G
    that round below zero are clamped to 0.
    """
    w, W = np.linalg.eigh(0.5 * (G + G.T))
    w = np.maximum(w, 0.0)
    return (W * (alpha * phi(alpha * w))) @ W.T


# --------------------------------------------------------------------------
# Section 3.1: matrix exponential-vector products
# --------------------------------------------------------------------------

def lowrank_exp_apply(H, alpha, X):
    """Y = exp(alpha H H^T) X by Theorem 3.1, following Algorithm 2's preprocessing.

    Step 2: skinny QR H = Q R.  Step 3: SVD R = U Sigma V^T.  Step 4: Q~ = Q U,
    D = Sigma^2.  Product (Remark after Theorem 3.1, steps (i)-(v)):
        Y = Q~ exp(alpha D) (Q~^T X) + X - Q~ (Q~^T X).
    H is d x m, X is d x b (natural numpy matrices).
    """
    Q, R = np.linalg.qr(H, mode="reduced")
    U, s, _ = np.linalg.svd(R)
    Qt = Q @ U
    D = s * s
    W = Qt.T @ X
    return Qt @ (np.exp(alpha * D)[:, None] * W) + X - Qt @ W


def dense_exp_apply(H, alpha, X, route="taylor"):
    """Y = exp(alpha H H^T) X with the d x d exponential formed densely (Algorithm 1, step 1)."""
    S = alpha * (H @ H.T)
    if route == "taylor":
        E = expm_taylor(S)
    else:
        E = sym_fun(S, np.exp, route=route)
    return E @ X


def scale_c2(lmax_w, lmax_b, tau):
    """Data scale c^2 = tau / max(lambda_max(H_W^T H_W), lambda_max(H_B^T H_B)).

    The paper normalises samples (Section 4) so that both spectra stay small;
    the synthetic workloads instead fix tau = c^2 * max(lambda_max) so that
    the top eigenvalue of M is at most e^tau.
    """
    m = max(float(lmax_w), float(lmax_b))
    if m <= 0.0:
        raise ValueError("both scatter matrices vanish")
    return tau / m


def m_apply(HW, HB, c2, X):
    """w = M v for M of Eq. (3.15), as the three products (iii)-(v) of Eq. (3.16)."""
    Y = lowrank_exp_apply(HW, -0.5 * c2, X)
    Y = lowrank_exp_apply(HB, c2, Y)
    return lowrank_exp_apply(HW, -0.5 * c2, Y)


def n_apply(HW, HB, c2, X):
    """w = exp(-c^2 S_W) exp(c^2 S_B) v, the nonsymmetric operator of Eq. (3.1) (Section 3.1), as the
    two Theorem 3.1 products of Algorithm 2's Arnoldi branch (steps 6A-10A: exp(c^2 S_B) first, then
    exp(-c^2 S_W))."""
    Y = lowrank_exp_apply(HB, c2, X)
    return lowrank_exp_apply(HW, -c2, Y)


def eda_arnoldi(HW, HB, t, c2, tol=1e-10, m_max=None, seed=0):
    """t dominant eigenpairs of exp(-c^2 S_W) exp(c^2 S_B) x = lambda x (Eq. (3.1)) by the Arnoldi
    method (Section 3.1), with no recovery step: the Ritz vectors are the x of Eq. (1.7) directly.

    From a seeded unit start vector v_1: w = N v_j (n_apply), orthogonalised against v_1 .. v_j by
    modified Gram-Schmidt, applied twice, the coefficients summed into column j of the upper
    Hessenberg H; h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}. After each step the Ritz pairs
    (theta, V_j s) come from the eigenpairs of H_j (numpy.linalg.eig), taken by decreasing real part,
    and the residual of a unit Ritz vector is h_{j+1,j} |e_j^T s| (the Arnoldi relation); the method
    stops once the t largest have residual <= tol |theta|, or when w vanishes (an invariant
    subspace). N - I maps into span([H_W, H_B]), so the space is exhausted after at most n + k + 1
    steps (the default m_max). N is similar to the symmetric M (N = E_W^{-1/2} M E_W^{1/2}), so its
    eigenvalues are real; the real parts are returned. Returns lam_t (descending), X_t (unit Ritz
    vectors), V = orth(X_t), the residuals and the number of steps.
    """
    d = HW.shape[0]
    if m_max is None:
        m_max = min(d, HW.shape[1] + HB.shape[1] + 1)
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(d)
    Vb = np.zeros((d, m_max + 1))
    Hh = np.zeros((m_max + 1, m_max))
    Vb[:, 0] = v / np.linalg.norm(v)
    best = None
    for j in range(m_max):
        w = n_apply(HW, HB, c2, Vb[:, j:j + 1])[:, 0]
        for _ in range(2):
            for i in range(j + 1):
                hij = Vb[:, i] @ w
                Hh[i, j] += hij
                w = w - hij * Vb[:, i]
        hnext = np.linalg.norm(w)
        m = j + 1
        theta, S = np.linalg.eig(Hh[:m, :m])
        order = np.argsort(-theta.real, kind="stable")[: min(t, m)]
        th = theta[order].real
        Sm = S[:, order]
        # a real eigenvector for each (real) Ritz value: remove the phase of its largest entry
        piv = np.argmax(np.abs(Sm), axis=0)
        Sm = (Sm * np.exp(-1j * np.angle(Sm[piv, np.arange(Sm.shape[1])]))).real
        Sm = Sm / np.linalg.norm(Sm, axis=0)
        res = hnext * np.abs(Sm[m - 1, :])
        best = (th, Vb[:, :m] @ Sm, res, m)
        done = m >= t and np.all(res <= tol * np.abs(th))
        if done or hnext <= 1e-14 * max(1.0, np.abs(Hh[:m, :m]).max()) or m == m_max:
            break
        Hh[m, j] = hnext
        Vb[:, m] = w / hnext
    th, Xt, res, m = best
    return dict(lam_t=th, Xt=Xt, V=orth(Xt), relres=res / np.abs(th), steps=m)


# --------------------------------------------------------------------------
# Section 3: the symmetric eigenproblem My = lambda y and its solution
# --------------------------------------------------------------------------

def orth(Xt):
    """Orthonormal basis of span(Xt) via Householder QR (Algorithm 3, step 6)."""
    Q, _ = np.linalg.qr(Xt, mode="reduced")
    return Q


def _solve_small(SW, SB, t, c2, route):
    """Steps shared by both tiers on (small or full) symmetric S_W, S_B.

    E_W^{-1/2} = exp(-c^2 S_W / 2) (Eq. (3.11)), E_B = exp(c^2 S_B) (Eq. (3.9)),
    M = E_W^{-1/2} E_B E_W^{-1/2} (Eq. (3.15)); the t largest eigenpairs
    (lambda, y) of M (Eq. (3.13)), x = E_W^{-1/2} y (Eq. (3.14)).
    """
    EWmh = sym_fun(c2 * SW, lambda w: np.exp(-0.5 * w), route=route)
    EB = sym_fun(c2 * SB, np.exp, route=route)
    M = EWmh @ EB @ EWmh
    M = 0.5 * (M + M.T)
    if route == "jacobi":
        lam, Y = jacobi_eigh(M)
    else:
        lam, Y = np.linalg.eigh(M)
    order = np.argsort(-lam, kind="stable")
    lam = lam[order]
    Y = Y[:, order]
    Xt = EWmh @ Y[:, :t]
    return lam, Y, Xt


def eda_dense(HW, HB, t, c2, route="eigh"):
    """Tier A: the dense EDA of Algorithm 1 in the symmetric form of Eq. (3.13).

    Forms S_W = H_W H_W^T and S_B = H_B H_B^T (Eqs. (1.1), (1.2)) as d x d
    matrices. Returns lam (all d eigenvalues of M, descending), Y_t, X_t and
    V = orth(X_t).
    """
    SW = HW @ HW.T
    SB = HB @ HB.T
    lam, Y, Xt = _solve_small(SW, SB, t, c2, route)
    return dict(lam=lam, lam_t=lam[:t].copy(), Y=Y[:, :t], Xt=Xt, V=orth(Xt))


def eda_projected(HW, HB, t, c2, route="eigh"):
    """Tier B: the same problem restricted to span([H_W, H_B]).

    Q from the Householder QR of Z = [H_W, H_B] spans a space that contains the
    ranges of S_W and S_B; on its orthogonal complement both vanish and M is
    the identity (Theorem 3.1 with f(0) = exp(0) = 1). So with R_W = Q^T H_W and
    R_B = Q^T H_B the eigenpairs of M above 1 are those of the (n+k)-dimensional
    M_r built from A_W = R_W R_W^T and A_B = R_B R_B^T, lifted by Q.
    lam lists the eigenvalues of M_r followed by d - (n+k) ones.
    """
    d = HW.shape[0]
    Z = np.concatenate([HW, HB], axis=1)
    Q, _ = np.linalg.qr(Z, mode="reduced")
    RW = Q.T @ HW
    RB = Q.T @ HB
    lam_r, Yr, Xr = _solve_small(RW @ RW.T, RB @ RB.T, t, c2, route)
    extra = max(d - Q.shape[1], 0)
    lam = np.sort(np.concatenate([lam_r, np.ones(extra)]))[::-1]
    Xt = Q @ Xr
    return dict(lam=lam, lam_t=lam_r[:t].copy(), Y=Q @ Yr[:, :t], Xt=Xt, V=orth(Xt), lam_r=lam_r)


def eda(X, labels, k, t, tau=None, c2=None, tier="auto"):
    """Algorithm 3 solved exactly: build H_W, H_B, fix c^2, solve, orthonormalise.

    Exactly one of tau (scale target) and c2 (explicit scale) is given.
    tier: "dense" (tier A), "projected" (tier B) or "auto" (dense for d <= 512).
    """
    f = scatter_factors(X, labels, k)
    HW, HB = f["HW"], f["HB"]
    lmax_w = float(np.linalg.eigvalsh(gram(HW))[-1])
    lmax_b = float(np.linalg.eigvalsh(gram(HB))[-1])
    if c2 is None:
        c2 = scale_c2(lmax_w, lmax_b, tau)
    d = HW.shape[0]
    if tier == "auto":
        tier = "dense" if d <= 512 else "projected"
    sol = eda_dense(HW, HB, t, c2) if tier == "dense" else eda_projected(HW, HB, t, c2)
    sol.update(f)
    sol.update(c2=c2, lmax_w=lmax_w, lmax_b=lmax_b, tier=tier)
    return sol


def eda_cholesky_route(HW, HB, t, c2):
    """Second route for the pencil (exp(c^2 S_B), exp(c^2 S_W)) of Eq. (1.7) (small d only).

    E_W = L L^T (Cholesky); the eigenvalues of L^{-1} E_B L^{-T} are those of the
    pencil. The exponentials come from the Taylor route, not from an
    eigendecomposition.
    """
    EW = expm_taylor(c2 * (HW @ HW.T))
    EB = expm_taylor(c2 * (HB @ HB.T))
    L = np.linalg.cholesky(0.5 * (EW + EW.T))
    Li = np.linalg.inv(L)
    C = Li @ EB @ Li.T
    C = 0.5 * (C + C.T)
    lam, Z = jacobi_eigh(C)
    order = np.argsort(-lam, kind="stable")
    lam = lam[order]
    Xg = Li.T @ Z[:, order[:t]]       # generalized eigenvectors x
    return dict(lam=lam, lam_t=lam[:t].copy(), Xt=Xg, V=orth(Xg))


def trace_ratio(V, HW, HB, c2):
    """rho(V) = tr((V^T exp(c^2 S_W) V)^{-1} (V^T exp(c^2 S_B) V)), Eq. (1.6), small d only."""
    EW = sym_fun(c2 * (HW @ HW.T), np.exp)
    EB = sym_fun(c2 * (HB @ HB.T), np.exp)
    return float(np.trace(np.linalg.solve(V.T @ EW @ V, V.T @ EB @ V)))


# --------------------------------------------------------------------------
# Section 3.3: projection, nearest-neighbour classification, subspace angle
# --------------------------------------------------------------------------

def project(V, X):
    """P = V^T X for samples given as (m, d) rows; returns (m, t) (Section 3.3, d_ij definition)."""
    return np.asarray(X, dtype=np.float64) @ V


def nn_classify(Ptrain, ytrain, Ptest):
    """1-NN with the L2 metric (Section 4): label of the nearest projected training sample.

    Squared distances are summed from coordinate differences; ties go to the
    smaller training index. Returns (labels, nearest distance, margin), the
    margin being the distance to the nearest sample of another class minus the
    nearest distance.
    """
    m = Ptest.shape[0]
    pred = np.empty(m, dtype=np.int32)
    dmin = np.empty(m)
    margin = np.empty(m)
    for j in range(m):
        diff = Ptrain - Ptest[j][None, :]
        dist = np.sqrt(np.sum(diff * diff, axis=1))
        i = int(np.argmin(dist))          # first minimum = smallest index
        pred[j] = ytrain[i]
        dmin[j] = dist[i]
        other = dist[np.asarray(ytrain) != ytrain[i]]
        margin[j] = (other.min() - dist[i]) if other.size else np.inf
    return pred, dmin, margin


def sin_angle(V, Vt):
    """sin of the largest principal angle, ||(I - V V^T) Vt||_2 (Theorem 3.8), V and Vt orthonormal."""
    R = Vt - V @ (V.T @ Vt)
    return float(np.linalg.norm(R, 2))
