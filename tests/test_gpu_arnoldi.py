"""Arnoldi-EDA on the GPU (eda_solve_arnoldi, the nonsymmetric form of Eq. (3.1)) against the oracle.

The operator exp(-c^2 S_W) exp(c^2 S_B) is checked element by element against the oracle's two Theorem 3.1
products (n_apply, Algorithm 2 steps 6A-10A through the paper's QR / SVD route). The solve is checked
against the oracle's exact symmetric route (the pencil of Eq. (1.7) has the same eigenvalues and
generalized eigenvectors, N being similar to M) and against the oracle's own Arnoldi method on small
problems: eigenvalues within 1e-10 (tau = 10; the attainable 64 eps lambda_1 / lambda_i at tau = 20),
the subspace of the generalized eigenvectors within 1e-8 (the residual bound at tau = 20), identical 1-NN
labels on the held-out samples.
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


@pytest.mark.parametrize("prec_name", ["f64", "tc"])
@pytest.mark.parametrize("d,k,nj,b,tau", [
    (256, 8, 6, 1, 10.0),
    (777, 9, [2, 5, 3, 4, 6, 2, 3, 7, 1], 5, 10.0),      # ragged d
    (4096, 40, 5, 40, 10.0),                              # 40 columns: two narrow blocks of the sweeps
    (600, 300, 1, 3, 10.0),                               # n_j = 1 (Example 1.1): H_W = 0, n > 256 with k = n
])
def test_n_apply_matches_oracle(eda, prec_name, d, k, nj, b, tau):
    p = synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=700 + d)
    f = O.scatter_factors(p.X, p.labels, p.k)
    c2 = _oracle_c2(f, tau)
    rng = np.random.default_rng(d + b)
    Xb = rng.standard_normal((d, b))
    Yr = O.n_apply(f["HW"], f["HB"], c2, Xb)
    prec = eda.EDA_F64 if prec_name == "f64" else eda.EDA_F64_TC
    with eda.build(_dev(p.X), _dev(p.labels), p.k, eda.config(prec=prec, block_b=2, tau=tau, tc_min_mi=-1)) as h:
        assert abs(h.c2 - c2) <= 1e-13 * c2
        Y = h.apply_exp(eda.OP_N, _dev(Xb.T)).cpu().numpy().T
    assert _colwise(Y, Yr) <= 1e-12, _colwise(Y, Yr)


def _solve(eda, p, t, b, tau, tol, prec):
    cfg = eda.config(prec=prec, block_b=b, tau=tau, tc_min_mi=-1)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
        V, lam, info, code = h.solve_arnoldi(t, tol, relres=True)
        assert code == 0, info
        Ptr = h.project(V, _dev(p.X)).cpu().numpy() if p.Xtest.shape[0] else None
        Pte = h.project(V, _dev(p.Xtest)).cpu().numpy() if p.Xtest.shape[0] else None
        c2 = h.c2
    return c2, lam.cpu().numpy(), V.cpu().numpy().T, info, Ptr, Pte


def _compare(p, t, tau, c2, lam, V, info, Ptr, Pte, tier):
    ref = O.eda(p.X, p.labels, p.k, t, tau=tau, tier=tier)
    assert abs(c2 - ref["c2"]) <= 1e-13 * ref["c2"]
    rel = np.abs(lam - ref["lam_t"]) / ref["lam_t"]
    floor = 64 * EPS * ref["lam_t"][0] / ref["lam_t"]
    assert np.all(rel <= np.maximum(1e-10, floor)), rel.max()
    assert np.abs(V.T @ V - np.eye(t)).max() <= 1e-12
    s = O.sin_angle(ref["V"], V)
    if Ptr is not None:
        lab_g, _, _ = O.nn_classify(Ptr, p.labels, Pte)
        lab_o, _, _ = O.nn_classify(O.project(ref["V"], p.X), p.labels, O.project(ref["V"], p.Xtest))
        assert np.array_equal(lab_g, lab_o)
    return ref, s


@pytest.mark.parametrize("prec_name", ["f64", "tc"])
def test_arnoldi_small_matches_oracle_arnoldi(eda, prec_name):
    # the oracle's own Arnoldi method (Section 3.1) and its exact dense route on a ragged problem, b = 1 and 3
    p = synth.gaussian_clusters(d=333, k=7, n_per_class=[2, 3, 5, 1, 4, 3, 2], seed=55, n_test_per_class=2)
    prec = eda.EDA_F64 if prec_name == "f64" else eda.EDA_F64_TC
    f = O.scatter_factors(p.X, p.labels, p.k)
    c2 = _oracle_c2(f, 8.0)
    ra = O.eda_arnoldi(f["HW"], f["HB"], p.k - 1, c2, tol=1e-13)
    for b in (1, 3):
        c2g, lam, V, info, Ptr, Pte = _solve(eda, p, p.k - 1, b, 8.0, 1e-12, prec)
        ref, s = _compare(p, p.k - 1, 8.0, c2g, lam, V, info, Ptr, Pte, "dense")
        assert s <= 1e-8, s
        assert np.allclose(lam, ra["lam_t"], rtol=1e-10, atol=0)
        assert O.sin_angle(ra["V"], V) <= 1e-8


@pytest.mark.parametrize("prec_name", ["f64", "tc"])
@pytest.mark.parametrize("name,tol", [("d256_k8", 1e-12), ("d4096_k40", 1e-12), ("d16384_k100", 1e-10)])
def test_arnoldi_matches_oracle(eda, prec_name, name, tol):
    c = synth.CONFIGS[name]
    p = synth.config_problem(name)
    prec = eda.EDA_F64 if prec_name == "f64" else eda.EDA_F64_TC
    c2, lam, V, info, Ptr, Pte = _solve(eda, p, c["t"], c["b"], c["tau"], tol, prec)
    ref, s = _compare(p, c["t"], c["tau"], c2, lam, V, info, Ptr, Pte, "auto" if p.d <= 512 else "projected")
    if c["tau"] <= 10.0:
        assert s <= 1e-8, s
    else:
        # per-vector residual bound over the gap to lambda_{t+1} = 1, plus the FP64 rounding floor of both routes
        t = c["t"]
        gap = ref["lam_t"][t - 1] - 1.0
        rr = np.asarray(info["relres"]) * lam
        dk = np.sqrt(np.sum((rr / np.maximum(lam - 1.0, gap)) ** 2))
        assert s <= dk + 64 * EPS * np.sqrt(t) * ref["lam_t"][0] / gap, (s, dk)
