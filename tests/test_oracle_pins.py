"""Pins for the FP64 oracle: closed forms, invariants and brute force from the paper.

Each test checks an oracle function against something other than itself: a
value fixed by the mathematics or by the paper's theorems. A plausible slip
in the oracle (a dropped term, a sign, a transposed operand, a wrong index or
summation order) fails at least one of these.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1512_06500_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_sym(rng, m, scale=1.0):
    A = rng.standard_normal((m, m)) * scale
    return 0.5 * (A + A.T)


def _known_spectrum(rng, w):
    """Q diag(w) Q^T with Q a product of two explicit Householder reflectors."""
    m = len(w)
    u = rng.standard_normal(m); u /= np.linalg.norm(u)
    v = rng.standard_normal(m); v /= np.linalg.norm(v)
    Q = (np.eye(m) - 2 * np.outer(u, u)) @ (np.eye(m) - 2 * np.outer(v, v))
    return Q @ np.diag(w) @ Q.T, Q


# ------------------------------------------------------------------ Section 1

def test_segment_brute_force_and_stability():
    rng = np.random.default_rng(1)
    k = 7
    labels = rng.integers(0, k, size=200).astype(np.int32)
    labels[:k] = np.arange(k)                      # no empty class
    counts, offsets, perm = O.segment(labels, k)
    for j in range(k):
        members = [i for i in range(labels.size) if labels[i] == j]
        assert counts[j] == len(members)
        assert list(perm[offsets[j]:offsets[j + 1]]) == members    # class-major, input order
    assert offsets[0] == 0 and offsets[-1] == labels.size
    assert sorted(perm.tolist()) == list(range(labels.size))


@pytest.mark.parametrize("bad", [[0, 1, 3], [0, -1, 2], [0, 0, 2]])
def test_segment_rejects_bad_labels(bad):
    with pytest.raises(ValueError):
        O.segment(np.array(bad), 3)


def test_scatter_factors_exact_means_and_identities():
    p = synth.gaussian_clusters(d=16, k=4, n_per_class=[1, 3, 5, 2], seed=3)
    f = O.scatter_factors(p.X, p.labels, p.k)
    n, d = p.X.shape
    # centroids equal the exact rational means up to the rounding of the running sum
    for j in range(p.k):
        idx = [i for i in range(n) if p.labels[i] == j]
        for q in range(d):
            exact = sum(Fraction(float(p.X[i, q])) for i in idx) / len(idx)
            assert abs(float(exact) - f["mu_j"][j, q]) <= 8 * np.finfo(float).eps * max(1.0, abs(float(exact)))
    for q in range(d):
        exact = sum(Fraction(float(v)) for v in p.X[:, q]) / n
        assert abs(float(exact) - f["mu"][q]) <= 8 * np.finfo(float).eps
    # H_W columns of one class sum to zero; sum_j sqrt(n_j) H_B[:, j] = sum_j n_j (mu_j - mu) = 0
    HW, HB = f["HW"], f["HB"]
    for j in range(p.k):
        cols = HW[:, f["offsets"][j]:f["offsets"][j + 1]]
        assert np.abs(cols.sum(axis=1)).max() < 1e-14
    s = HB @ np.sqrt(f["counts"].astype(float))
    assert np.abs(s).max() < 1e-13
    # S_W + S_B equals the total scatter sum_i (chi_i - mu)(chi_i - mu)^T
    C = p.X.T - f["mu"][:, None]
    assert np.allclose(HW @ HW.T + HB @ HB.T, C @ C.T, atol=1e-12)
    # column p of H_W is sample perm[p] minus its own class mean
    for q in range(n):
        i = f["perm"][q]
        assert np.array_equal(HW[:, q], p.X[i] - f["mu_j"][p.labels[i]])


def test_scatter_factors_summation_order_is_input_order():
    # values whose sum depends on the order: 1e16 + 1 - 1e16
    X = np.zeros((3, 1))
    X[:, 0] = [1e16, 1.0, -1e16]
    f = O.scatter_factors(X, np.array([0, 0, 0]), 1)
    assert f["mu"][0] == ((0.0 + 1e16) + 1.0 + -1e16) / 3.0
    assert f["mu"][0] == 0.0       # 1e16 + 1 rounds to 1e16


# ------------------------------------------------------------------ Section 2

def test_jacobi_closed_forms():
    w, U = O.jacobi_eigh(np.diag([3.0, -1.0, 2.0]))
    assert np.allclose(w, [-1.0, 2.0, 3.0])
    a, b, c = 2.0, 1.0, 5.0
    w, U = O.jacobi_eigh(np.array([[a, b], [b, c]]))
    disc = math.sqrt(((a - c) / 2) ** 2 + b * b)
    assert np.allclose(w, [(a + c) / 2 - disc, (a + c) / 2 + disc], rtol=0, atol=1e-14)


def test_jacobi_known_spectrum():
    rng = np.random.default_rng(2)
    w0 = np.array([-2.0, -0.5, 0.0, 0.0, 1e-3, 1.0, 4.0, 9.0])
    A, _ = _known_spectrum(rng, w0)
    w, U = O.jacobi_eigh(A)
    assert np.allclose(w, np.sort(w0), atol=1e-13)
    assert np.allclose(U.T @ U, np.eye(8), atol=1e-13)
    assert np.allclose(A @ U, U * w, atol=1e-13)


def test_expm_taylor_closed_forms():
    assert np.array_equal(O.expm_taylor(np.zeros((4, 4))), np.eye(4))
    D = np.diag([-3.0, 0.0, 0.5, 7.0])
    assert np.allclose(O.expm_taylor(D), np.diag(np.exp([-3.0, 0.0, 0.5, 7.0])), rtol=1e-14, atol=0)
    th = 2.3
    R = O.expm_taylor(np.array([[0.0, th], [-th, 0.0]]))
    assert np.allclose(R, [[math.cos(th), math.sin(th)], [-math.sin(th), math.cos(th)]], atol=1e-14)
    rng = np.random.default_rng(4)
    A = _rand_sym(rng, 6, 1.5)
    assert np.allclose(O.expm_taylor(A) @ O.expm_taylor(-A), np.eye(6), atol=1e-12)


def test_exp_eigen_routes_agree_with_taylor():
    rng = np.random.default_rng(5)
    A = _rand_sym(rng, 10, 2.0)
    E = O.expm_taylor(A)
    scale = np.abs(E).max()
    assert np.abs(O.sym_fun(A, np.exp, "eigh") - E).max() < 1e-13 * scale
    assert np.abs(O.sym_fun(A, np.exp, "jacobi") - E).max() < 1e-13 * scale


def test_phi_and_phi_operator_series():
    assert O.phi(np.array([0.0]))[0] == 1.0
    z = np.array([1e-12, -3e-9, 0.7, -5.0])
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    # the defining series summed in 40-digit arithmetic
    ref = np.array([float(mpmath.nsum(lambda j: mpmath.mpf(x) ** j / mpmath.factorial(j + 1), [0, mpmath.inf]))
                    for x in z])
    assert np.allclose(O.phi(z), ref, rtol=4e-16, atol=0)
    rng = np.random.default_rng(6)
    H = rng.standard_normal((9, 5))
    G = H.T @ H
    G /= np.linalg.eigvalsh(G)[-1]
    for alpha in (1.0, -0.5, -3.0):
        ser = np.zeros_like(G)
        term = np.eye(5)                      # alpha^j G^(j-1) / j!, j = 1..
        for j in range(1, 60):
            ser += alpha ** j * term / math.factorial(j)
            term = term @ G
        assert np.abs(O.phi_operator(G, alpha) - ser).max() < 1e-14 * max(1.0, np.abs(ser).max())


def test_phi_operator_doubling_identity():
    """K(alpha) = alpha phi(alpha G) (Theorem 3.1) obeys K(2 alpha) = K(alpha) (2 I + G K(alpha)): from
    phi(2 z) = phi(z) (1 + e^z) / 2 and e^(alpha G) = I + G K(alpha). A slip in phi (a dropped 1/z,
    e^z for expm1), in the clamping of tiny eigenvalues or in the scaling by alpha breaks it."""
    rng = np.random.default_rng(23)
    for m, r in ((7, 7), (12, 5)):                       # full rank and rank deficient (null space)
        H = rng.standard_normal((30, r)) @ rng.standard_normal((r, m))
        G = H.T @ H
        G /= np.linalg.eigvalsh(G)[-1]
        for alpha in (0.3, -0.5, 2.0, -4.0):
            K1 = O.phi_operator(G, alpha)
            K2 = O.phi_operator(G, 2 * alpha)
            rhs = K1 @ (2 * np.eye(m) + G @ K1)
            assert np.abs(K2 - rhs).max() <= 1e-13 * np.abs(K2).max(), (m, alpha)


# ---------------------------------------------------------------- Section 3.1

@pytest.mark.parametrize("alpha", [1.0, -0.5, -1.0])
def test_theorem_3_1_low_rank_identity(alpha):
    rng = np.random.default_rng(7)
    d, m, b = 40, 9, 3
    H = rng.standard_normal((d, m)) * 0.25
    X = rng.standard_normal((d, b))
    Y_ref = O.dense_exp_apply(H, alpha, X, route="taylor")
    Y = O.lowrank_exp_apply(H, alpha, X)
    assert np.linalg.norm(Y - Y_ref) / np.linalg.norm(Y_ref) < 1e-13
    # the phi form of the same identity: exp(alpha H H^T) = I + H K(alpha) H^T
    Yk = X + H @ (O.phi_operator(H.T @ H, alpha) @ (H.T @ X))
    assert np.linalg.norm(Yk - Y_ref) / np.linalg.norm(Y_ref) < 1e-13


def test_theorem_3_1_rank_deficient_and_zero():
    rng = np.random.default_rng(8)
    d = 30
    B = rng.standard_normal((d, 3))
    H = np.concatenate([B, B @ rng.standard_normal((3, 4))], axis=1) * 0.3   # rank 3, 7 columns
    X = rng.standard_normal((d, 2))
    Y_ref = O.dense_exp_apply(H, -1.0, X)
    assert np.linalg.norm(O.lowrank_exp_apply(H, -1.0, X) - Y_ref) < 1e-13 * np.linalg.norm(Y_ref)
    Z = np.zeros((d, 5))
    assert np.array_equal(O.lowrank_exp_apply(Z, 2.0, X), X)        # exp(0) = I
    assert np.array_equal(O.phi_operator(np.zeros((4, 4)), 2.5), 2.5 * np.eye(4))


def test_m_apply_matches_dense_symmetric_form():
    rng = np.random.default_rng(9)
    p = synth.gaussian_clusters(d=24, k=3, n_per_class=3, seed=9)
    f = O.scatter_factors(p.X, p.labels, p.k)
    c2 = 0.3
    X = rng.standard_normal((24, 2))
    EWmh = O.expm_taylor(-0.5 * c2 * f["HW"] @ f["HW"].T)
    EB = O.expm_taylor(c2 * f["HB"] @ f["HB"].T)
    ref = EWmh @ EB @ EWmh @ X
    assert np.linalg.norm(O.m_apply(f["HW"], f["HB"], c2, X) - ref) < 1e-12 * np.linalg.norm(ref)


def test_composed_form_of_the_three_products():
    """M - I = Z C Z^T with Z = [H_W H_B] (Theorem 3.1 applied to each factor of the symmetric form):
    the small-space recurrence the library's composed M-apply follows, written out here in numpy from
    G_W, G_WB = H_W^T H_B, K_W = K(-c^2/2) and K_B = K(c^2), equals the three products; and so does
    folding K into the factor, X + (H K)(H^T X)."""
    rng = np.random.default_rng(33)
    p = synth.gaussian_clusters(d=60, k=4, n_per_class=[3, 5, 2, 4], seed=33)
    f = O.scatter_factors(p.X, p.labels, p.k)
    HW, HB = f["HW"], f["HB"]
    c2 = 0.7
    KW = O.phi_operator(O.gram(HW), -0.5 * c2)
    KB = O.phi_operator(O.gram(HB), c2)
    GW, GWB = HW.T @ HW, HW.T @ HB
    Y = rng.standard_normal((60, 3))
    pw, qb = HW.T @ Y, HB.T @ Y
    u1 = KW @ pw                       # y1 = y + H_W u1
    q1 = qb + GWB.T @ u1               # H_B^T y1
    p1 = pw + GW @ u1                  # H_W^T y1
    v = KB @ q1                        # y2 = y1 + H_B v
    p2 = p1 + GWB @ v                  # H_W^T y2
    u3 = KW @ p2                       # M y = y2 + H_W u3
    composed = Y + HW @ (u1 + u3) + HB @ v
    ref = O.m_apply(HW, HB, c2, Y)
    assert np.linalg.norm(composed - ref) <= 1e-13 * np.linalg.norm(ref)
    folded = Y + (HW @ KW) @ (HW.T @ Y)
    assert np.linalg.norm(folded - O.lowrank_exp_apply(HW, -0.5 * c2, Y)) <= 1e-13 * np.linalg.norm(folded)


# ---------------------------------------------------------------- Section 3.2/3.3

def test_commuting_diagonal_closed_form():
    # H_W and H_B supported on shared coordinate axes: S_W = diag(w), S_B = diag(b)
    d = 12
    w = np.array([0.5, 2.0, 0.0, 1.0, 3.0])
    b = np.array([4.0, 1.0, 2.5, 0.0, 0.2])
    HW = np.zeros((d, 5)); HB = np.zeros((d, 5))
    for i in range(5):
        HW[i, i] = math.sqrt(w[i]); HB[i, i] = math.sqrt(b[i])
    c2 = 0.7
    expect = np.sort(np.concatenate([np.exp(c2 * (b - w)), np.ones(d - 5)]))[::-1]
    t = 2                                  # b_i - w_i > 0 for exactly two axes
    for sol in (O.eda_dense(HW, HB, t, c2), O.eda_dense(HW, HB, t, c2, route="jacobi"),
                O.eda_projected(HW, HB, t, c2)):
        assert np.allclose(sol["lam"], expect, rtol=1e-13, atol=0)
        top = np.argsort(-(b - w))[:t]
        E = np.zeros((d, t)); E[top, np.arange(t)] = 1.0
        assert O.sin_angle(E, sol["V"]) < 1e-12


# ---------------------------------------------------------------- Section 3.1, Eq. (3.1): Arnoldi form

def test_n_apply_matches_dense_product():
    # N X = exp(-c^2 S_W) exp(c^2 S_B) X by two Theorem 3.1 products against the dense Taylor exponentials
    p = synth.gaussian_clusters(d=40, k=3, n_per_class=[4, 2, 5], seed=21)
    f = O.scatter_factors(p.X, p.labels, p.k)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((40, 3))
    c2 = 0.4
    dense = O.dense_exp_apply(f["HW"], -c2, O.dense_exp_apply(f["HB"], c2, X))
    got = O.n_apply(f["HW"], f["HB"], c2, X)
    assert np.abs(got - dense).max() <= 1e-12 * np.abs(dense).max()


@pytest.mark.parametrize("spec", [(90, 4, [5, 3, 6, 4], 12), (150, 6, 3, 13), (64, 2, [7, 1], 14)])
def test_arnoldi_eda_matches_symmetric_route(spec):
    # N = E_W^{-1/2} M E_W^{1/2} (Eq. (3.1) against the symmetric form of Section 3.2): the same
    # eigenvalues, and x = E_W^{-1/2} y, so the same span of the t eigenvectors
    d, k, nj, seed = spec
    p = synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=seed)
    f = O.scatter_factors(p.X, p.labels, p.k)
    HW, HB = f["HW"], f["HB"]
    c2 = O.scale_c2(np.linalg.eigvalsh(O.gram(HW))[-1], np.linalg.eigvalsh(O.gram(HB))[-1], 10.0)
    t = k - 1
    ref = O.eda_dense(HW, HB, t, c2)
    a = O.eda_arnoldi(HW, HB, t, c2)
    assert np.all(np.abs(a["lam_t"] - ref["lam_t"]) <= 1e-10 * ref["lam_t"])
    assert O.sin_angle(ref["V"], a["V"]) <= 1e-8
    assert a["steps"] <= HW.shape[1] + HB.shape[1] + 1


def test_arnoldi_eda_commuting_closed_form():
    # the diagonal factors of test_commuting_diagonal_closed_form: lambda = exp(c^2 (b_i - w_i)), axes
    d = 12
    w = np.array([0.5, 2.0, 0.0, 1.0, 3.0])
    b = np.array([4.0, 1.0, 2.5, 0.0, 0.2])
    HW = np.zeros((d, 5)); HB = np.zeros((d, 5))
    for i in range(5):
        HW[i, i] = math.sqrt(w[i]); HB[i, i] = math.sqrt(b[i])
    c2 = 0.7
    t = 2
    a = O.eda_arnoldi(HW, HB, t, c2, m_max=d)
    expect = np.sort(np.exp(c2 * (b - w)))[::-1][:t]
    assert np.allclose(a["lam_t"], expect, rtol=1e-12, atol=0)
    top = np.argsort(-(b - w))[:t]
    E = np.zeros((d, t)); E[top, np.arange(t)] = 1.0
    assert O.sin_angle(E, a["V"]) < 1e-10


def test_arnoldi_eda_full_spectrum_tiny():
    # full-rank factors of a 6-dimensional problem: the Arnoldi method run to m = d returns every
    # eigenvalue of the dense nonsymmetric N
    rng = np.random.default_rng(31)
    d = 6
    HW = 0.6 * rng.standard_normal((d, d))
    HB = 0.8 * rng.standard_normal((d, 3))
    c2 = 0.5
    N = O.dense_exp_apply(HW, -c2, O.dense_exp_apply(HB, c2, np.eye(d)))
    ev = np.sort(np.linalg.eigvals(N).real)[::-1]
    a = O.eda_arnoldi(HW, HB, d, c2, tol=0.0, m_max=d)
    assert a["steps"] == d
    assert np.allclose(a["lam_t"], ev, rtol=1e-11, atol=0)


def _load_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, val = line.split(":", 1)
            out[key.strip()] = [float(v) for v in val.split()]
    return out


def test_example_1_1_golden():
    g = _load_golden("example_1_1.txt")
    d, k = int(g["d"][0]), int(g["k"][0])
    X = np.array(g["X_rows"]).reshape(d, d)
    labels = np.array(g["labels"], dtype=np.int32)
    f = O.scatter_factors(X, labels, k)
    assert np.array_equal(f["HW"], np.zeros((d, d)))                 # H_W = O
    sol = O.eda_dense(f["HW"], f["HB"], 3, g["c2"][0])
    assert np.allclose(sol["lam"], g["lambda"], rtol=1e-14, atol=0)
    u = np.array(g["unit_eigvec_for_lambda_1"])
    assert abs(abs(u @ sol["Y"][:, 2]) - 1.0) < 1e-13                 # eigenvector 1/sqrt(3) (1,1,1)


def test_example_1_1_general_n_equals_k():
    # n_j = 1 for all classes: H_W = O and the eigenvalues are exp(c^2 mu_i(G_B))
    rng = np.random.default_rng(11)
    d, k = 10, 5
    X = rng.standard_normal((k, d))
    f = O.scatter_factors(X, np.arange(k), k)
    c2 = 0.4
    mu = np.linalg.eigvalsh(f["HB"].T @ f["HB"])
    expect = np.sort(np.concatenate([np.exp(c2 * np.maximum(mu, 0)), np.ones(d - k)]))[::-1]
    sol = O.eda_dense(f["HW"], f["HB"], k - 1, c2)
    assert np.allclose(sol["lam"], expect, rtol=1e-13, atol=1e-13)
    assert np.sum(sol["lam"] > 1 + 1e-9) == k - 1


def _random_problem(d, k, nj, seed, tau=3.0):
    p = synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=seed)
    f = O.scatter_factors(p.X, p.labels, p.k)
    lw = np.linalg.eigvalsh(f["HW"].T @ f["HW"])[-1]
    lb = np.linalg.eigvalsh(f["HB"].T @ f["HB"])[-1]
    return p, f, O.scale_c2(lw, lb, tau)


def test_theorem_3_7_unit_eigenvalue_count():
    d, k, nj = 40, 4, 4
    p, f, c2 = _random_problem(d, k, nj, seed=12)
    n = k * nj
    lam = O.eda_dense(f["HW"], f["HB"], k - 1, c2)["lam"]
    delta = 1e-9 * lam[0]
    assert np.sum(np.abs(lam - 1) <= delta) >= d - n + 1                  # Theorem 3.7
    # sharper count for affinely independent samples (rank S_B = k-1, rank S_W = n-k)
    assert np.sum(lam > 1 + delta) == k - 1
    assert np.sum(np.abs(lam - 1) <= delta) == d - n + 1
    assert np.sum(lam < 1 - delta) == n - k


def test_theorem_3_3_bounds():
    d = 20
    p, f, c2 = _random_problem(d, 3, 3, seed=13)
    lam = O.eda_dense(f["HW"], f["HB"], 2, c2)["lam"]
    nu = np.sort(np.linalg.eigvalsh(c2 * f["HW"] @ f["HW"].T))[::-1]     # nu_1 >= ... >= nu_d
    mu = np.sort(np.linalg.eigvalsh(c2 * f["HB"] @ f["HB"].T))[::-1]
    for i in range(d):
        lo = max(math.exp(mu[i] - nu[0]), math.exp(mu[d - 1] - nu[d - 1 - i]))
        hi = min(math.exp(mu[i] - nu[d - 1]), math.exp(mu[0] - nu[d - 1 - i]))
        assert lo * (1 - 1e-12) <= lam[i] <= hi * (1 + 1e-12)


def test_lemma_3_4_theorem_3_5_trace_ratio():
    d, t = 16, 3
    p, f, c2 = _random_problem(d, 4, 3, seed=14)
    sol = O.eda_dense(f["HW"], f["HB"], t, c2)
    rho = O.trace_ratio(sol["Xt"], f["HW"], f["HB"], c2)
    assert abs(rho - sol["lam_t"].sum()) < 1e-11 * rho
    # invariance under V -> V R and the maximality of the top eigenvectors
    rng = np.random.default_rng(15)
    R = rng.standard_normal((t, t))
    assert abs(O.trace_ratio(sol["Xt"] @ R, f["HW"], f["HB"], c2) - rho) < 1e-10 * rho
    Vr = O.orth(rng.standard_normal((d, t)))
    assert O.trace_ratio(Vr, f["HW"], f["HB"], c2) <= rho * (1 + 1e-12)
    nu = np.sort(np.linalg.eigvalsh(c2 * f["HW"] @ f["HW"].T))[::-1]
    mu = np.sort(np.linalg.eigvalsh(c2 * f["HB"] @ f["HB"].T))[::-1]
    lo = sum(max(math.exp(mu[d - t + i] - nu[0]), math.exp(mu[d - 1] - nu[t - i - 1])) for i in range(t))
    hi = sum(min(math.exp(mu[i] - nu[d - 1]), math.exp(mu[0] - nu[d - 1 - i])) for i in range(t))
    assert lo * (1 - 1e-12) <= rho <= hi * (1 + 1e-12)


def test_brute_force_tiny_cholesky_route():
    for d, k, nj, seed in [(6, 2, 2, 16), (8, 3, 2, 17)]:
        p, f, c2 = _random_problem(d, k, nj, seed)
        t = k - 1
        a = O.eda_dense(f["HW"], f["HB"], t, c2)
        b = O.eda_cholesky_route(f["HW"], f["HB"], t, c2)
        j = O.eda_dense(f["HW"], f["HB"], t, c2, route="jacobi")
        assert np.allclose(a["lam"], b["lam"], rtol=1e-13, atol=0)
        assert np.allclose(a["lam"], j["lam"], rtol=1e-13, atol=0)
        assert O.sin_angle(a["V"], b["V"]) < 1e-11
        assert O.sin_angle(a["V"], j["V"]) < 1e-11
        # the generalized eigenvectors satisfy exp(c2 S_B) x = lambda exp(c2 S_W) x
        EW = O.expm_taylor(c2 * f["HW"] @ f["HW"].T)
        EB = O.expm_taylor(c2 * f["HB"] @ f["HB"].T)
        for i in range(t):
            x = a["Xt"][:, i]
            r = EB @ x - a["lam_t"][i] * (EW @ x)
            assert np.linalg.norm(r) < 1e-12 * a["lam_t"][i] * np.linalg.norm(EW @ x)


@pytest.mark.parametrize("d", [64, 256])
def test_tier_a_equals_tier_b(d):
    p, f, c2 = _random_problem(d, 6, 4, seed=18 + d, tau=10.0)
    t = 5
    a = O.eda_dense(f["HW"], f["HB"], t, c2)
    b = O.eda_projected(f["HW"], f["HB"], t, c2)
    assert np.allclose(a["lam"], b["lam"], rtol=1e-11, atol=0)
    assert O.sin_angle(a["V"], b["V"]) < 1e-9


def _gap_bound(lam_all, t, lam1):
    """The subspace tolerance of two FP64 routes: eps lambda_1 over the gap lambda_t - lambda_{t+1}
    (lambda_{t+1} = 1, Theorem 3.7), times a safety factor for the d-dimensional products."""
    gap = lam_all[t - 1] - lam_all[t]
    return 1e3 * np.finfo(float).eps * lam1 / gap


@pytest.mark.parametrize("d,k,nj", [(1024, 20, 5), (4096, 40, 5)])
def test_tier_a_equals_tier_b_large(d, k, nj):
    # the projected route (tier B) carries every GPU parity check at d >= 4096; here it is held to the
    # dense definition (tier A: d x d scatter matrices, their exponentials and M formed explicitly) at
    # the benchmark's d = 4096 and at 1024, on the benchmark's kind of problem (t = k - 1)
    p, f, c2 = _random_problem(d, k, nj, seed=d + 1, tau=10.0)
    t = k - 1
    a = O.eda_dense(f["HW"], f["HB"], t, c2)
    b = O.eda_projected(f["HW"], f["HB"], t, c2)
    rel = np.abs(a["lam_t"] - b["lam_t"]) / b["lam_t"]
    assert rel.max() <= 1e-12, rel.max()
    # every eigenvalue of M, not only the wanted ones: d - (n + k) ones and the n + k of the projection
    assert np.abs(a["lam"] - b["lam"]).max() <= 1e-12 * b["lam"][0]
    assert O.sin_angle(a["V"], b["V"]) <= _gap_bound(b["lam"], t, b["lam"][0])


@pytest.mark.parametrize("d", [64, 96])
def test_jacobi_route_equals_eigh_route(d):
    # the oracle's default symmetric eigen route (LAPACK eigh) against its own cyclic Jacobi sweeps,
    # through the whole dense solve (three eigendecompositions: E_W^{-1/2}, E_B and M)
    p, f, c2 = _random_problem(d, 6, 4, seed=40 + d, tau=10.0)
    t = 5
    a = O.eda_dense(f["HW"], f["HB"], t, c2, route="jacobi")
    b = O.eda_dense(f["HW"], f["HB"], t, c2, route="eigh")
    assert np.abs(a["lam"] - b["lam"]).max() <= 1e-12 * b["lam"][0]
    assert O.sin_angle(a["V"], b["V"]) <= _gap_bound(b["lam"], t, b["lam"][0])


def test_scale_c2_hand_values():
    # c^2 = tau / max(lambda_max(G_W), lambda_max(G_B)) (reading A1), by hand
    assert O.scale_c2(4.0, 2.5, 10.0) == 2.5
    assert O.scale_c2(1.0, 8.0, 20.0) == 2.5
    assert O.scale_c2(0.0, 5.0, 10.0) == 2.0
    with pytest.raises(ValueError):
        O.scale_c2(0.0, 0.0, 10.0)


@pytest.mark.parametrize("w_max,b_max", [(1.0, 4.0), (4.0, 1.0)])
def test_scale_c2_sets_theorem_3_3_bound(w_max, b_max):
    # Commuting factors on disjoint coordinates: S_W = diag(w) on the first axes, S_B = diag(b) on the
    # next ones. Then M = exp(c^2 S_B) exp(-c^2 S_W) is diagonal and lambda_1(M) = e^{c^2 max b}
    # (Theorem 3.3 with nu_d = 0: lambda_1 <= e^{c^2 mu_1}, attained here). With the scale rule,
    # c^2 max(w_max, b_max) = tau, so lambda_1 = e^tau exactly when the between-class Gram dominates
    # and e^{tau b_max / w_max} below it otherwise. Using min instead of max, or tau * lambda_max,
    # changes lambda_1 by orders of magnitude.
    d, tau = 16, 6.0
    w = np.array([w_max, 0.5, 0.25])
    b = np.array([b_max, 0.75, 0.1])
    HW = np.zeros((d, 3))
    HB = np.zeros((d, 3))
    for i in range(3):
        HW[i, i] = np.sqrt(w[i])
        HB[3 + i, i] = np.sqrt(b[i])
    lw = np.linalg.eigvalsh(O.gram(HW))[-1]
    lb = np.linalg.eigvalsh(O.gram(HB))[-1]
    c2 = O.scale_c2(lw, lb, tau)
    sol = O.eda_dense(HW, HB, 2, c2)
    expect = math.exp(tau * b_max / max(w_max, b_max))
    assert abs(sol["lam"][0] - expect) <= 1e-12 * expect
    assert sol["lam"][0] <= math.exp(tau) * (1 + 1e-12)


def test_scale_c2_example_1_1_tight():
    # n_j = 1 (Example 1.1): H_W = 0, so lambda_max(G_W) = 0, c^2 = tau / lambda_max(G_B) and the top
    # eigenvalue of M is e^{c^2 lambda_max(G_B)} = e^tau exactly
    rng = np.random.default_rng(41)
    d, k, tau = 24, 5, 7.0
    X = rng.standard_normal((k, d))
    lab = np.arange(k, dtype=np.int32)
    sol = O.eda(X, lab, k, k - 1, tau=tau, tier="dense")
    assert sol["lmax_w"] == 0.0
    assert abs(sol["lam"][0] - math.exp(tau)) <= 1e-12 * math.exp(tau)


def _angle_pair(rng, d, theta):
    """Orthonormal V, Vt (d x t) whose principal angles are exactly theta: V = Q_1 R_1 and
    Vt = (Q_1 diag(cos theta) + Q_2 diag(sin theta)) R_2 with [Q_1 Q_2] orthonormal and R_1, R_2
    random rotations (so V^T Vt is not symmetric)."""
    t = len(theta)
    Q, _ = np.linalg.qr(rng.standard_normal((d, 2 * t)))
    R1, _ = np.linalg.qr(rng.standard_normal((t, t)))
    R2, _ = np.linalg.qr(rng.standard_normal((t, t)))
    V = Q[:, :t] @ R1
    Vt = (Q[:, :t] * np.cos(theta) + Q[:, t:] * np.sin(theta)) @ R2
    return V, Vt


def test_sin_angle_known_principal_angles():
    # Theorem 3.8 measures the subspace error by the sine of the largest principal angle,
    # ||(I - V V^T) Vt||_2. On a pair with prescribed angles it must return max sin(theta_i).
    rng = np.random.default_rng(42)
    theta = np.array([1e-9, 1e-5, 0.3, 1.3, 0.8])
    V, Vt = _angle_pair(rng, 40, theta)
    expect = np.sin(theta).max()
    assert abs(O.sin_angle(V, Vt) - expect) <= 1e-15
    assert abs(O.sin_angle(Vt, V) - expect) <= 1e-15        # symmetric in its arguments
    # tiny angles, which 1 - cos cannot resolve: the direct formula keeps them
    theta = np.array([1e-12, 3e-10, 2e-9])
    V, Vt = _angle_pair(rng, 30, theta)
    assert abs(O.sin_angle(V, Vt) - np.sin(2e-9)) <= 1e-6 * 2e-9
    # the same span in another basis: angle 0
    V, _ = _angle_pair(rng, 30, np.zeros(4))
    R, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    assert O.sin_angle(V, V @ R) <= 1e-15


def test_sin_angle_pin_rejects_plausible_slips():
    # mistakes planted in copies of the oracle's formula (on the CPU): the prescribed-angle pin above
    # rejects each of them by far
    rng = np.random.default_rng(43)
    theta = np.array([0.05, 0.2, 0.6])
    V, Vt = _angle_pair(rng, 25, theta)
    expect = np.sin(theta).max()
    transposed = float(np.linalg.norm(Vt - V @ (Vt.T @ V), 2))          # (V^T Vt)^T in place of V^T Vt
    frobenius = float(np.linalg.norm(Vt - V @ (V.T @ Vt)))              # Frobenius in place of the 2-norm
    cosines = float(np.sqrt(max(0.0, 1 - np.linalg.svd(V.T @ Vt, compute_uv=False).max() ** 2)))  # smallest angle
    for wrong in (transposed, frobenius, cosines):
        assert abs(wrong - expect) > 1e-2, wrong
    assert abs(O.sin_angle(V, Vt) - expect) <= 1e-15


def test_scale_invariance():
    p = synth.gaussian_clusters(d=32, k=4, n_per_class=3, seed=19)
    a = O.eda(p.X, p.labels, p.k, 3, tau=5.0)
    b = O.eda(3.0 * p.X, p.labels, p.k, 3, tau=5.0)
    assert abs(b["c2"] * 9.0 - a["c2"]) < 1e-14 * a["c2"]
    assert np.allclose(a["lam_t"], b["lam_t"], rtol=1e-12, atol=0)
    assert O.sin_angle(a["V"], b["V"]) < 1e-10


# ---------------------------------------------------------------- Section 3.3 / 4

def test_nn_classify_brute_force():
    Ptr = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0], [1.0, 0.0]])
    ytr = np.array([0, 1, 2, 3])
    Pte = np.array([[0.9, 0.1], [0.5, 0.0], [0.0, 1.6]])
    pred, dmin, margin = O.nn_classify(Ptr, ytr, Pte)
    assert pred.tolist() == [1, 0, 2]      # (0.5, 0) ties samples 0 and 1 -> smaller index
    assert abs(dmin[0] - math.hypot(0.1, 0.1)) < 1e-15
    assert margin[1] == 0.0


def test_theorem_3_8_distance_bound():
    rng = np.random.default_rng(20)
    d, t = 30, 4
    V = O.orth(rng.standard_normal((d, t)))
    Vt = O.orth(V + 1e-3 * rng.standard_normal((d, t)))
    s = O.sin_angle(V, Vt)
    c = math.sqrt(max(1 - s * s, 0.0))
    for _ in range(50):
        x = rng.standard_normal(d); x /= np.linalg.norm(x)
        y = rng.standard_normal(d); y /= np.linalg.norm(y)
        dd = np.linalg.norm(V.T @ (x - y))
        dt = np.linalg.norm(Vt.T @ (x - y))
        assert (dt - 2 * s) / c <= dd + 1e-14
        assert dd <= dt * c + 2 * s + 1e-14
