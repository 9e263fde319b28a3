"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Integer and centroid outputs are compared bit for bit. Floating-point results of the FP64 path
are held to the FP64 targets: eigenvalues within 1e-10 relative, the largest principal angle of
the t-dimensional subspace within 1e-8, identical 1-NN labels. Operator-level results
(Gram, K(alpha), exp-vector products) are compared with tolerances derived from FP64 rounding:
with unit roundoff u = 1.1e-16, a length-L dot product carries at most about L u of relative
error, so products over d <= 4096 rows and n <= 200 columns stay below 1e-12 relative to the
norms involved.
"""
import numpy as np
import pytest

import oracle as O
from paper_1512_06500_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(float).eps


@pytest.fixture(scope="module")
def eda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_06500_gb300 import build_lib, eda as E
    build_lib.build()
    E.load()
    return E


DEV = "cuda:0"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _problem(d, k, nj, seed, test=0):
    return synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=seed, n_test_per_class=test)


# ----------------------------------------------------------------- build step (bit-exact)

@pytest.mark.parametrize("d,k,nj,dtype", [
    (256, 8, 6, np.float64),
    (300, 5, [1, 4, 7, 2, 3], np.float64),       # ragged d, uneven classes incl. n_j = 1
    (1000, 33, 3, np.float32),                    # FP32 input, k > 32 (several scatter rounds)
])
def test_build_bitexact(eda, d, k, nj, dtype):
    p = _problem(d, k, nj, seed=100 + d)
    X = p.X.astype(dtype)
    ref = O.scatter_factors(X.astype(np.float64), p.labels, p.k)
    with eda.build(_dev(X), _dev(p.labels), p.k, eda.config(block_b=2)) as h:
        f = h.factors()
        assert np.array_equal(f["counts"].cpu().numpy(), ref["counts"])
        assert np.array_equal(f["perm"].cpu().numpy(), ref["perm"])
        assert np.array_equal(f["HW"].cpu().numpy().T, ref["HW"])
        assert np.array_equal(f["HB"].cpu().numpy().T, ref["HB"])


def test_gram_eigen_and_phi_operator(eda):
    p = _problem(512, 12, 5, seed=7)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, eda.config(block_b=4, tau=10.0)) as h:
        f = h.factors()
        ref = O.scatter_factors(p.X, p.labels, p.k)
        GW = O.gram(ref["HW"])
        GB = O.gram(ref["HB"])
        assert np.abs(f["GW"].cpu().numpy() - GW).max() <= 64 * 512 * EPS * np.abs(GW).max()
        assert np.abs(f["GB"].cpu().numpy() - GB).max() <= 64 * 512 * EPS * np.abs(GB).max()
        # eigenvalues: absolute accuracy of a backward-stable solver, n u ||G||
        ew = np.sort(np.linalg.eigvalsh(GW))
        assert np.abs(f["evals_w"].cpu().numpy() - ew).max() <= 64 * 60 * EPS * ew[-1]
        assert abs(h.lmax_w - ew[-1]) <= 64 * EPS * ew[-1]
        c2 = O.scale_c2(ew[-1], np.linalg.eigvalsh(GB)[-1], 10.0)
        assert abs(h.c2 - c2) <= 1e-13 * c2
        KW = O.phi_operator(GW, -0.5 * c2)
        KB = O.phi_operator(GB, c2)
        assert np.abs(f["KW"].cpu().numpy() - KW).max() <= 1e-12 * np.abs(KW).max()
        assert np.abs(f["KB"].cpu().numpy() - KB).max() <= 1e-12 * np.abs(KB).max()


# ----------------------------------------------------------------- exp-vector products

def _oracle_c2(ref, tau):
    """c^2 from the oracle's own Grams (reading A1), never from the library."""
    lw = float(np.linalg.eigvalsh(O.gram(ref["HW"]))[-1])
    lb = float(np.linalg.eigvalsh(O.gram(ref["HB"]))[-1])
    return O.scale_c2(lw, lb, tau)


def _colwise(Y, Yr):
    """max over columns j of max_i |Y - Yr|_ij / max_i |Yr|_ij: an error confined to a few rows (a tile
    edge at a ragged d) cannot hide under a norm of the whole block."""
    return float(np.max(np.abs(Y - Yr).max(axis=0) / np.abs(Yr).max(axis=0)))


@pytest.mark.parametrize("d,k,nj,b", [(256, 8, 6, 1), (777, 9, [2, 5, 3, 4, 6, 2, 3, 7, 1], 5), (4096, 40, 5, 8),
                                      (1000, 9, [2, 5, 3, 4, 6, 2, 3, 7, 1], 33)])
def test_apply_exp_matches_theorem_3_1(eda, d, k, nj, b):
    # element by element against the oracle's product through the paper's own QR / SVD route
    # (Algorithm 2), with the oracle's own factors and scale; ragged d and block widths
    p = _problem(d, k, nj, seed=200 + d)
    rng = np.random.default_rng(d)
    Xb = rng.standard_normal((d, b))
    ref = O.scatter_factors(p.X, p.labels, p.k)
    c2 = _oracle_c2(ref, 10.0)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, eda.config(block_b=2, tau=10.0)) as h:
        assert abs(h.c2 - c2) <= 1e-13 * c2
        Xt = _dev(Xb.T)
        # the library's alpha selects its stored operators (the first two) or forms K(alpha) anew
        for op, H, a_lib, a_ref in [(eda.OP_SW, ref["HW"], -0.5 * h.c2, -0.5 * c2), (eda.OP_SB, ref["HB"], h.c2, c2),
                                    (eda.OP_SW, ref["HW"], 0.8 * c2, 0.8 * c2),
                                    (eda.OP_SB, ref["HB"], -1.3 * c2, -1.3 * c2)]:
            Y = h.apply_exp(op, Xt, alpha=a_lib).cpu().numpy().T
            Yr = O.lowrank_exp_apply(H, a_ref, Xb)
            err = _colwise(Y, Yr)
            assert err <= 1e-12, (op, a_ref, err)
        Y = h.apply_exp(eda.OP_M, Xt).cpu().numpy().T
        Yr = O.m_apply(ref["HW"], ref["HB"], c2, Xb)
        assert _colwise(Y, Yr) <= 1e-12


def test_apply_exp_zero_factor_is_identity(eda):
    # all samples of each class identical: H_W = 0, exp(alpha S_W) X = X exactly
    d, k = 64, 4
    rng = np.random.default_rng(3)
    means = rng.random((k, d))
    labels = np.repeat(np.arange(k), 3).astype(np.int32)
    X = means[labels]
    with eda.build(_dev(X), _dev(labels), k, eda.config(block_b=1, c2=0.5)) as h:
        Xb = rng.standard_normal((2, d))
        Y = h.apply_exp(eda.OP_SW, _dev(Xb), alpha=-0.25).cpu().numpy()
        assert np.array_equal(Y, Xb)


def test_single_class_has_no_between_class_scatter(eda):
    # k = 1: H_B = sqrt(n)(mu_1 - mu) = 0, so exp(alpha S_B) X = X exactly, and c^2 comes from G_W alone
    d, n = 300, 9
    rng = np.random.default_rng(12)
    X = rng.random((n, d))
    labels = np.zeros(n, dtype=np.int32)
    with eda.build(_dev(X), _dev(labels), 1, eda.config(tau=10.0)) as h:
        Xb = rng.standard_normal((3, d))
        Y = h.apply_exp(eda.OP_SB, _dev(Xb), alpha=h.c2).cpu().numpy()
        assert np.array_equal(Y, Xb)
        # the eigensolver resolves the 1 x 1 zero Gram to an absolute ~1e-19, negligible in c^2 (A1)
        assert h.lmax_b <= 1e-15 * h.lmax_w
        lw = float(np.linalg.eigvalsh(O.gram(O.scatter_factors(X, labels, 1)["HW"]))[-1])
        assert abs(h.c2 - 10.0 / lw) <= 1e-12 * (10.0 / lw)


@pytest.mark.parametrize("tau", [1.0, 10.0, 40.0])
def test_phi_by_squaring_matches_oracle(eda, tau):
    # n, k <= 256: lambda_max by the Lanczos run and K(alpha) by scaling and squaring (no eigenvectors);
    # tau sets how many doublings each side takes. K against the oracle's eigenpair form (Theorem 3.1)
    p = _problem(700, 9, [20, 25, 18, 30, 22, 19, 27, 21, 24], seed=71)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, eda.config(block_b=4, tau=tau)) as h:
        f = h.factors()
        ref = O.scatter_factors(p.X, p.labels, p.k)
        GW, GB = O.gram(ref["HW"]), O.gram(ref["HB"])
        lw, lb = np.linalg.eigvalsh(GW)[-1], np.linalg.eigvalsh(GB)[-1]
        assert abs(h.lmax_w - lw) <= 64 * EPS * lw
        assert abs(h.lmax_b - lb) <= 64 * EPS * lb
        c2 = O.scale_c2(lw, lb, tau)
        assert abs(h.c2 - c2) <= 1e-13 * c2
        for key, G, a in (("KW", GW, -0.5 * c2), ("KB", GB, c2)):
            K = O.phi_operator(G, a)
            assert np.abs(f[key].cpu().numpy() - K).max() <= 1e-12 * np.abs(K).max(), key


@pytest.mark.parametrize("gap", [0.0, 1e-9, 1e-3])
def test_lanczos_lambda_max_clustered_top(eda, gap):
    # H_W with prescribed singular values: a top eigenvalue of G_W that is double (gap 0), nearly double
    # (the Lanczos bounds may not certify it: the eigensolver's value is taken) or separated
    rng = np.random.default_rng(17)
    d, n, k = 400, 60, 5
    Qd, _ = np.linalg.qr(rng.standard_normal((d, n)))
    Pn, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = np.linspace(0.2, 0.9, n)
    sig[-1], sig[-2] = 1.0, np.sqrt(1.0 - gap)
    HW = (Qd * sig) @ Pn.T
    HB = 0.3 * rng.standard_normal((d, k))
    with eda.build_from_factors(_dev(HW.T), _dev(HB.T), eda.config(block_b=2, tau=10.0)) as h:
        assert abs(h.lmax_w - 1.0) <= 64 * EPS
        lb = np.linalg.eigvalsh(HB.T @ HB)[-1]
        assert abs(h.lmax_b - lb) <= 64 * EPS * lb


# ----------------------------------------------------------------- full solve

def _solve_and_compare(eda, p, t, b, tau, tol=1e-12, tier="auto", check_every=1, m_form=0):
    cfg = eda.config(block_b=b, tau=tau, check_every=check_every, true_residuals=1, m_form=m_form)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
        V, lam, Y, info, code = h.solve(t, tol, want_y=True, relres=True)
        assert code == 0, info
        ref = O.eda(p.X, p.labels, p.k, t, tau=tau, tier=tier)
        assert abs(h.c2 - ref["c2"]) <= 1e-13 * ref["c2"]
        lam = lam.cpu().numpy()
        rel = np.abs(lam - ref["lam_t"]) / ref["lam_t"]
        assert rel.max() <= 1e-10, rel.max()
        Vg = V.cpu().numpy().T
        assert np.abs(Vg.T @ Vg - np.eye(t)).max() <= 1e-12
        s = O.sin_angle(ref["V"], Vg)
        assert s <= 1e-8, s
        assert info["max_relres_true"] <= max(10 * tol, 1e-12), info
        # 1-NN on the projected held-out samples: identical labels
        if p.Xtest.shape[0]:
            Ptr = h.project(V, _dev(p.X)).cpu().numpy()
            Pte = h.project(V, _dev(p.Xtest)).cpu().numpy()
            Ptr_ref = O.project(ref["V"], p.X)
            Pte_ref = O.project(ref["V"], p.Xtest)
            # the projection itself, with the same V, against the oracle's product
            assert np.abs(Pte - O.project(Vg, p.Xtest)).max() <= 1e-12 * np.abs(Pte).max()
            lab_g, _, _ = O.nn_classify(Ptr, p.labels, Pte)
            lab_o, _, margin = O.nn_classify(Ptr_ref, p.labels, Pte_ref)
            assert np.array_equal(lab_g, lab_o)
        return info, lam, ref


def test_solve_d256_k8_b1(eda):
    c = synth.CONFIGS["d256_k8"]
    p = synth.config_problem("d256_k8")
    _solve_and_compare(eda, p, c["t"], c["b"], c["tau"])


def test_solve_d4096_k40_b8(eda):
    c = synth.CONFIGS["d4096_k40"]
    p = synth.config_problem("d4096_k40")
    info, lam, ref = _solve_and_compare(eda, p, c["t"], c["b"], c["tau"])
    assert info["basis_cols"] <= p.n + p.k + c["b"]


@pytest.mark.parametrize("b,check_every", [(1, 3), (3, 2), (5, 1), (40, 1)])
def test_solve_ragged_blocks(eda, b, check_every):
    # b = 40 is wider than the sample count (n = 20): most of every block lies inside the basis and is
    # refilled with fresh directions
    # block size that does not divide t, uneven classes, d not a multiple of any tile
    p = _problem(333, 7, [2, 3, 5, 1, 4, 3, 2], seed=55, test=2)
    _solve_and_compare(eda, p, p.k - 1, b, 8.0, check_every=check_every)


@pytest.mark.parametrize("spec", [(300, 4, [3, 2, 4, 3], 900), (512, 3, [5, 2, 7], 902),
                                  (777, 6, [2, 3, 4, 2, 3, 5], 903)])
def test_solve_every_block_size_small_problems(eda, spec):
    # n + k <= 25: the block Krylov space is exhausted within a few blocks and, at some block sizes, a
    # column of a new block is nearly dependent on the others; its content can drop below the rounding
    # of the block's Gram and be replaced by a fresh direction. The pairs must still be those of the
    # oracle, with true FP64 residuals at the tolerance (the solver verifies and refines after refills)
    d, k, nj, seed = spec
    p = synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=seed, n_test_per_class=2)
    t = k - 1
    ref = None
    for b in list(range(1, 13)) + [16]:
        cfg = eda.config(block_b=b, tau=10.0, true_residuals=1)
        with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
            if ref is None:
                ref = O.eda(p.X, p.labels, p.k, t, tau=10.0, tier="projected")
            assert abs(h.c2 - ref["c2"]) <= 1e-13 * ref["c2"]
            V, lam, _, info, code = h.solve(t, 1e-12, check=False)
            assert code == 0, (b, info)
            assert info["max_relres_true"] <= 1e-11, (b, info)
            rel = np.abs(lam.cpu().numpy() - ref["lam_t"]) / ref["lam_t"]
            assert rel.max() <= 1e-10, (b, rel.max())
            assert O.sin_angle(ref["V"], V.cpu().numpy().T) <= 1e-10, b


@pytest.mark.parametrize("name", ["d256_k8", "d4096_k40"])
def test_solve_composed_m_form(eda, name):
    # the same operator M in its composed form I + Z C Z^T (two sweeps over [H_W H_B]); the
    # independent true-residual check still uses the three products
    c = synth.CONFIGS[name]
    p = synth.config_problem(name)
    _solve_and_compare(eda, p, c["t"], c["b"], c["tau"], m_form=1)


def test_apply_m_composed_matches_three_products(eda):
    p = _problem(777, 9, [2, 5, 3, 4, 6, 2, 3, 7, 1], seed=31)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((6, 777))
    out = []
    for form in (0, 1):
        with eda.build(_dev(p.X), _dev(p.labels), p.k, eda.config(tau=8.0, m_form=form)) as h:
            out.append(h.apply_exp(eda.OP_M, _dev(X)).cpu().numpy())
    assert np.linalg.norm(out[1] - out[0]) <= 1e-13 * np.linalg.norm(out[0])


def test_solve_commuting_diagonal_closed_form(eda):
    d = 48
    w = np.array([0.5, 2.0, 0.0, 1.0, 3.0, 0.25])
    bb = np.array([4.0, 1.0, 2.5, 0.0, 0.2, 3.0])
    HW = np.zeros((d, 6))
    HB = np.zeros((d, 6))
    for i in range(6):
        HW[i, i] = np.sqrt(w[i])
        HB[i, i] = np.sqrt(bb[i])
    c2 = 0.7
    t = int(np.sum(bb - w > 0))
    expect = np.sort(np.exp(c2 * (bb - w)))[::-1][:t]
    with eda.build_from_factors(_dev(HW.T), _dev(HB.T), eda.config(block_b=2, c2=c2)) as h:
        V, lam, _, info, code = h.solve(t, 1e-13)
        assert code == 0
        assert np.allclose(lam.cpu().numpy(), expect, rtol=1e-12, atol=0)
        top = np.argsort(-(bb - w))[:t]
        E = np.zeros((d, t))
        E[top, np.arange(t)] = 1.0
        assert O.sin_angle(E, V.cpu().numpy().T) <= 1e-10


def test_example_1_1_one_sample_per_class(eda):
    # n_j = 1: H_W = O, lambda_i = exp(c^2 mu_i(G_B)) (Example 1.1)
    rng = np.random.default_rng(21)
    d, k = 40, 6
    X = rng.standard_normal((k, d))
    labels = np.arange(k, dtype=np.int32)
    with eda.build(_dev(X), _dev(labels), k, eda.config(block_b=1, tau=4.0)) as h:
        f = O.scatter_factors(X, labels, k)
        mu = np.sort(np.linalg.eigvalsh(f["HB"].T @ f["HB"]))[::-1][: k - 1]
        c2 = O.scale_c2(0.0, mu[0], 4.0)
        assert abs(h.c2 - c2) <= 1e-13 * c2
        V, lam, _, info, code = h.solve(k - 1, 1e-13)
        assert code == 0
        assert np.allclose(lam.cpu().numpy(), np.exp(c2 * mu), rtol=1e-11, atol=0)


# ----------------------------------------------------------------- error paths (host-detected)

def test_bad_labels_and_nonfinite(eda):
    p = _problem(64, 3, 3, seed=9)
    lab = p.labels.copy()
    lab[0] = 7
    with pytest.raises(eda.EdaError) as e:
        eda.build(_dev(p.X), _dev(lab), p.k)
    assert e.value.code == -2
    lab = np.array([0, 0, 2, 2, 0, 2, 0, 2, 0], dtype=np.int32)      # class 1 empty
    with pytest.raises(eda.EdaError) as e:
        eda.build(_dev(p.X), _dev(lab), 3)
    assert e.value.code == -2
    X = p.X.copy()
    X[4, 17] = np.nan
    with pytest.raises(eda.EdaError) as e:
        eda.build(_dev(X), _dev(p.labels), p.k)
    assert e.value.code == -3
    with pytest.raises(eda.EdaError) as e:
        eda.build(_dev(p.X), _dev(p.labels), p.n + 1)
    assert e.value.code == -1


def test_not_converged_is_reported(eda):
    p = synth.config_problem("d4096_k40")
    cfg = eda.config(block_b=8, tau=10.0, m_max=48)      # basis far too small for t = 39
    with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
        V, lam, _, info, code = h.solve(39, 1e-12, check=False)
        assert code == -8
        assert info["converged"] < 39
        assert np.all(np.isfinite(lam.cpu().numpy()))
