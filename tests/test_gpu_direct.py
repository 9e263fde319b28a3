"""The exact solve in the span of [H_W H_B] (eda_solve_direct) against the oracle and against eda_solve.

M - I = Z C Z^T with Z = [H_W H_B] (Theorem 3.1 for each factor of Eq. (3.15)), so the eigenpairs of M
above 1 are those of an (n - 1)-dimensional symmetric problem in the coordinates of Z (Theorem 3.7 for
the rest of the spectrum). The oracle solves the same problem densely (tier A) or after a Householder QR
of Z (tier B), sharing no code with the library. Bars as for the Krylov solvers: every eigenvalue within
max(1e-10, 64 eps lambda_1 / lambda_i) relative (reading A8), the subspace within 1e-8 at tau = 10 (at
tau = 20 within the FP64 rounding floor of both routes over the gap lambda_t - 1), identical 1-NN labels,
V orthonormal. Closed form: with one sample per class (Example 1.1) H_W = 0 and lambda_i = exp(c^2 mu_i(G_B)).
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


def _prec(eda, name):
    return eda.EDA_F64 if name == "f64" else eda.EDA_F64_TC


def _direct(eda, p, t, tau, prec, also_krylov=None):
    cfg = eda.config(prec=prec, block_b=8, tau=tau, tc_min_mi=-1)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
        V, lam, info, code = h.solve_direct(t)
        assert code == 0
        out = dict(c2=h.c2, lam=lam.cpu().numpy(), V=V.cpu().numpy().T, info=info)
        if p.Xtest.shape[0]:
            out["Ptr"] = h.project(V, _dev(p.X)).cpu().numpy()
            out["Pte"] = h.project(V, _dev(p.Xtest)).cpu().numpy()
        if also_krylov is not None:
            Vk, lamk, _, infok, codek = h.solve(t, also_krylov)
            assert codek == 0, infok
            out["lam_k"] = lamk.cpu().numpy()
            out["V_k"] = Vk.cpu().numpy().T
    return out


def _check(p, t, tau, g, tier, sin_bar=1e-8):
    ref = O.eda(p.X, p.labels, p.k, t, tau=tau, tier=tier)
    assert abs(g["c2"] - ref["c2"]) <= 1e-13 * ref["c2"]
    lam, V = g["lam"], g["V"]
    assert np.all(np.diff(lam) <= 0)
    rel = np.abs(lam - ref["lam_t"]) / ref["lam_t"]
    floor = 64 * EPS * ref["lam_t"][0] / ref["lam_t"]
    assert np.all(rel <= np.maximum(1e-10, floor)), (rel.max(), int(np.argmax(rel / np.maximum(1e-10, floor))))
    assert np.abs(V.T @ V - np.eye(t)).max() <= 1e-12
    s = O.sin_angle(ref["V"], V)
    if sin_bar is not None:
        assert s <= sin_bar, s
    if "Ptr" in g:
        lab_g, _, _ = O.nn_classify(g["Ptr"], p.labels, g["Pte"])
        lab_o, _, _ = O.nn_classify(O.project(ref["V"], p.X), p.labels, O.project(ref["V"], p.Xtest))
        assert np.array_equal(lab_g, lab_o), np.flatnonzero(lab_g != lab_o)
    return ref, s


@pytest.mark.parametrize("prec_name", ["f64", "tc"])
@pytest.mark.parametrize("name", ["d256_k8", "d4096_k40"])
def test_direct_matches_oracle(eda, prec_name, name):
    c = synth.CONFIGS[name]
    p = synth.config_problem(name)
    g = _direct(eda, p, c["t"], c["tau"], _prec(eda, prec_name), also_krylov=1e-10)
    _check(p, c["t"], c["tau"], g, "auto" if p.d <= 512 else "projected")
    # the Krylov solver on the same handle: the same eigenvalues and subspace
    assert np.allclose(g["lam"], g["lam_k"], rtol=1e-10, atol=0)
    assert O.sin_angle(g["V"], g["V_k"]) <= 1e-8


@pytest.mark.parametrize("prec_name", ["f64", "tc"])
def test_direct_ragged_matches_oracle(eda, prec_name):
    # ragged d (not a multiple of any tile), uneven classes including one of a single sample
    p = synth.gaussian_clusters(d=777, k=9, n_per_class=[2, 5, 3, 4, 6, 2, 3, 7, 1], seed=91, n_test_per_class=2)
    g = _direct(eda, p, p.k - 1, 10.0, _prec(eda, prec_name))
    _check(p, p.k - 1, 10.0, g, "dense")


@pytest.mark.parametrize("prec_name", ["f64", "tc"])
def test_direct_example_1_1_closed_form(eda, prec_name):
    # one sample per class (Example 1.1): H_W = 0, so M = exp(c^2 S_B) and lambda_i = exp(c^2 mu_i(G_B))
    k = 12
    p = synth.gaussian_clusters(d=300, k=k, n_per_class=1, seed=17)
    g = _direct(eda, p, k - 1, 10.0, _prec(eda, prec_name))
    f = O.scatter_factors(p.X, p.labels, p.k)
    mu = np.sort(np.linalg.eigvalsh(O.gram(f["HB"])))[::-1][: k - 1]
    expect = np.exp(g["c2"] * mu)
    assert np.allclose(g["lam"], expect, rtol=1e-11, atol=0), np.abs(g["lam"] / expect - 1).max()


def test_direct_d16384_k100(eda):
    c = synth.CONFIGS["d16384_k100"]
    p = synth.config_problem("d16384_k100")
    g = _direct(eda, p, c["t"], c["tau"], eda.EDA_F64_TC)
    _check(p, c["t"], c["tau"], g, "projected", sin_bar=1e-6)


def test_direct_dependent_samples_is_breakdown(eda):
    # two identical samples in one class make two columns of H_W equal: the kept columns are dependent
    p = synth.gaussian_clusters(d=200, k=4, n_per_class=3, seed=23, shuffle=False)
    X = p.X.copy()
    X[1] = X[0]
    with eda.build(_dev(X), _dev(p.labels), p.k, eda.config(prec=eda.EDA_F64, block_b=2, tau=10.0)) as h:
        _, _, _, code = h.solve_direct(3, check=False)
    assert code == -7   # EDA_ERR_BREAKDOWN


def test_direct_rejects_bad_arguments(eda):
    p = synth.gaussian_clusters(d=128, k=4, n_per_class=3, seed=29)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, eda.config(prec=eda.EDA_F64, block_b=2, tau=10.0)) as h:
        _, _, _, code = h.solve_direct(p.n, check=False)      # t > n - 1
        assert code == -1
    with eda.build(_dev(p.X), _dev(p.labels), p.k, eda.config(prec=eda.EDA_F32, block_b=2, tau=10.0)) as h:
        _, _, _, code = h.solve_direct(3, check=False)        # single-precision handle
        assert code == -1
