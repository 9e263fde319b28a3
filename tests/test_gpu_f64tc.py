"""The FP64 solver with its M-apply sweeps on the bf16 tensor cores (prec EDA_F64_TC) against the oracle.

The sweeps over Z = [H_W H_B] of the composed M-apply run as error-free split products (seven bf16 digit
planes per operand, exact integer accumulation); everything else is the FP64 solver. The tests force the
tensor-core products at every size (tc_min_mi = -1), below the size from which the library would pick them. The products are as
accurate as FP64 ones, so the FP64 bars apply unchanged: M-apply element by element within 1e-12 of the
column's largest entry (the oracle's three Theorem 3.1 products through its QR / SVD route), eigenvalues
within max(1e-10, 64 eps lambda_1 / lambda_i), the subspace within the Davis-Kahan bound of the residuals,
identical 1-NN labels.
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _colwise(Y, Yr):
    return float(np.max(np.abs(Y - Yr).max(axis=0) / np.abs(Yr).max(axis=0)))


def _oracle_c2(f, tau):
    lw = float(np.linalg.eigvalsh(O.gram(f["HW"]))[-1])
    lb = float(np.linalg.eigvalsh(O.gram(f["HB"]))[-1])
    return O.scale_c2(lw, lb, tau)


@pytest.mark.parametrize("d,k,nj,b,tau", [
    (256, 8, 6, 1, 10.0),
    (777, 9, [2, 5, 3, 4, 6, 2, 3, 7, 1], 5, 10.0),      # ragged d, n + k = 42
    (1000, 33, 5, 32, 10.0),                              # several 128-column bands of Z, one full narrow block
    (4096, 40, 5, 40, 10.0),                              # 40 columns: two narrow blocks
    (3000, 60, [3, 4] * 30, 17, 20.0),                    # tau = 20: lambda_1 ~ e^20
])
def test_m_apply_tc_matches_oracle(eda, d, k, nj, b, tau):
    p = synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=600 + d)
    f = O.scatter_factors(p.X, p.labels, p.k)
    c2 = _oracle_c2(f, tau)
    rng = np.random.default_rng(d + b)
    Xb = rng.standard_normal((d, b))
    Yr = O.m_apply(f["HW"], f["HB"], c2, Xb)
    out = {}
    for prec in (eda.EDA_F64_TC, eda.EDA_F64):
        cfg = eda.config(prec=prec, block_b=2, tau=tau, m_form=1, tc_min_mi=-1)
        with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
            assert abs(h.c2 - c2) <= 1e-13 * c2
            out[prec] = h.apply_exp(eda.OP_M, _dev(Xb.T)).cpu().numpy().T
    assert _colwise(out[eda.EDA_F64_TC], Yr) <= 1e-12, _colwise(out[eda.EDA_F64_TC], Yr)
    # and as close to the plain FP64 path as that path is to the oracle
    assert _colwise(out[eda.EDA_F64_TC], out[eda.EDA_F64]) <= 1e-12


def test_m_apply_tc_zero_and_constant_columns(eda):
    # degenerate digit planes: a zero block (all scales 0, every digit 0) gives exactly zero change, and a
    # block of constant columns (every digit of a row the same) is still reproduced
    p = synth.gaussian_clusters(d=500, k=6, n_per_class=4, seed=611)
    f = O.scatter_factors(p.X, p.labels, p.k)
    c2 = _oracle_c2(f, 8.0)
    cfg = eda.config(prec=eda.EDA_F64_TC, block_b=2, tau=8.0, tc_min_mi=-1)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
        Z = np.zeros((3, 500))
        Y = h.apply_exp(eda.OP_M, _dev(Z)).cpu().numpy()
        assert np.array_equal(Y, Z)
        C = np.ones((3, 500)) * np.array([[1.0], [-3.5], [1e-200]])
        Y = h.apply_exp(eda.OP_M, _dev(C)).cpu().numpy().T
        Yr = O.m_apply(f["HW"], f["HB"], c2, C.T)
        assert _colwise(Y, Yr) <= 1e-12


def test_m_apply_tc_extreme_magnitudes(eda):
    # the digit split reads mantissa and exponent from the bits: columns spanning 300 decades, subnormal
    # columns and one dominant entry over tiny ones are reproduced to 1e-12 of each column's largest entry
    p = synth.gaussian_clusters(d=700, k=7, n_per_class=5, seed=612)
    f = O.scatter_factors(p.X, p.labels, p.k)
    c2 = _oracle_c2(f, 10.0)
    rng = np.random.default_rng(613)
    sgn = lambda: rng.choice([-1.0, 1.0], size=700)
    X = np.empty((700, 3))
    X[:, 0] = sgn() * 10.0 ** rng.uniform(-150, 150, 700)
    X[:, 1] = sgn() * 10.0 ** rng.uniform(-318, -309, 700)       # subnormal entries only
    X[::5, 1] = 0.0
    X[:, 2] = sgn() * 1e-200
    X[17, 2] = 1e200
    cfg = eda.config(prec=eda.EDA_F64_TC, block_b=2, tau=10.0, tc_min_mi=-1)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
        Y = h.apply_exp(eda.OP_M, _dev(X.T)).cpu().numpy().T
    # the oracle on each column scaled by a power of two to a largest entry near 1 (exact in FP64, and M
    # is linear), so that its own products do not round in the subnormal range
    e = np.frexp(np.abs(X).max(axis=0))[1]
    Yr = np.ldexp(O.m_apply(f["HW"], f["HB"], c2, np.ldexp(X, -e[None, :])), e[None, :])
    assert np.all(np.isfinite(Y))
    assert _colwise(Y, Yr) <= 1e-12, _colwise(Y, Yr)


def _solve_compare(eda, p, t, b, tau, tol, ref):
    cfg = eda.config(prec=eda.EDA_F64_TC, block_b=b, tau=tau, true_residuals=1, tc_min_mi=-1)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
        assert abs(h.c2 - ref["c2"]) <= 1e-13 * ref["c2"]
        V, lam, _, info, code = h.solve(t, tol, relres=True)
        assert code == 0, info
        Ptr = h.project(V, _dev(p.X)).cpu().numpy()
        Pte = h.project(V, _dev(p.Xtest)).cpu().numpy()
    lam = lam.cpu().numpy()
    Vg = V.cpu().numpy().T
    lam_ref = ref["lam_t"]
    rel = np.abs(lam - lam_ref) / lam_ref
    floor = 64 * EPS * lam_ref[0] / lam_ref
    assert np.all(rel <= np.maximum(1e-10, floor)), rel.max()
    assert info["max_relres_true"] <= 10 * tol, info
    gap = lam_ref[t - 1] - 1.0
    rr = np.asarray(info["relres"]) * lam
    dk = np.sqrt(np.sum((rr / np.maximum(lam - 1.0, gap)) ** 2))
    kappa = np.exp(0.5 * ref["c2"] * ref["lmax_w"])
    s = O.sin_angle(ref["V"], Vg)
    assert s <= kappa * (dk + 64 * EPS * np.sqrt(t) * lam_ref[0] / gap), (s, dk)
    lab_g, _, _ = O.nn_classify(Ptr, p.labels, Pte)
    lab_o, _, _ = O.nn_classify(O.project(ref["V"], p.X), p.labels, O.project(ref["V"], p.Xtest))
    assert np.array_equal(lab_g, lab_o)
    return s, info


@pytest.mark.parametrize("name,tol", [("d256_k8", 1e-12), ("d4096_k40", 1e-12), ("d16384_k100", 1e-10)])
def test_solve_tc_matches_oracle(eda, name, tol):
    c = synth.CONFIGS[name]
    p = synth.config_problem(name)
    ref = O.eda(p.X, p.labels, p.k, c["t"], tau=c["tau"], tier="auto" if p.d <= 512 else "projected")
    s, info = _solve_compare(eda, p, c["t"], c["b"], c["tau"], tol, ref)
    if c["tau"] <= 10.0:
        assert s <= 1e-8


def test_solve_tc_ragged_small(eda):
    p = synth.gaussian_clusters(d=333, k=7, n_per_class=[2, 3, 5, 1, 4, 3, 2], seed=55, n_test_per_class=2)
    ref = O.eda(p.X, p.labels, p.k, p.k - 1, tau=8.0, tier="dense")
    for b in (1, 3, 5):
        s, _ = _solve_compare(eda, p, p.k - 1, b, 8.0, 1e-12, ref)
        assert s <= 1e-8


def test_solve_tc_d65536_k200_matches_oracle(eda):
    # the benchmark's workload and tolerance
    name = "d65536_k200"
    c = synth.CONFIGS[name]
    p = synth.config_problem(name)
    ref = O.eda(p.X, p.labels, p.k, c["t"], tau=c["tau"], tier="projected")
    s, info = _solve_compare(eda, p, c["t"], c["b"], c["tau"], 1e-6, ref)
    print(f"\nd65536_k200 (tensor-core FP64 sweeps): sin {s:.2e}, blocks {info['iters']}, refills {info['refills']}")


@pytest.mark.parametrize("d,k,nj", [(777, 9, [2, 5, 3, 4, 6, 2, 3, 7, 1]), (4096, 40, 5), (2000, 70, 4)])
def test_grams_tc_match_oracle(eda, d, k, nj):
    # the build's Grams as blocks of Z^T Z from the split Z: element by element within the FP64 bound of a
    # length-d dot product, exactly symmetric, and the cross Gram G_WB enters the composed M-apply (checked
    # above through M); n + k = 310 at the last size takes the eigenpair route for K
    p = synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=640 + d)
    f = O.scatter_factors(p.X, p.labels, p.k)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, eda.config(prec=eda.EDA_F64_TC, block_b=4, tau=10.0,
                                                                        tc_min_mi=-1)) as h:
        g = h.factors()
        for key, H in (("GW", f["HW"]), ("GB", f["HB"])):
            G = g[key].cpu().numpy()
            Gr = O.gram(H)
            assert np.array_equal(G, G.T), key
            assert np.abs(G - Gr).max() <= 64 * d * EPS * np.abs(Gr).max(), key
        c2 = _oracle_c2(f, 10.0)
        assert abs(h.c2 - c2) <= 1e-13 * c2
