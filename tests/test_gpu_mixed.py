"""Mixed-precision solver (single-precision H, basis and sweeps; FP64 small steps and FP64
refinement of the Ritz vectors) against the FP64 oracle.

Targets: eigenvalues within 1e-6 relative and identical 1-NN labels on held-out samples (the
mixed-precision bar), and, because the refinement runs until every true FP64 relative residual
is below tol, also the FP64 bar (1e-10 relative eigenvalues, principal angle 1e-8) when tol is
tight. The principal-angle bound follows from the residual: sin(angle) <= ||r|| / gap, with the
gap lambda_t - 1 read from the oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_1512_06500_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def _run(eda, p, t, b, tau, tol, prec):
    cfg = eda.config(prec=prec, block_b=b, tau=tau, true_residuals=1)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
        V, lam, _, info, code = h.solve(t, tol)
        assert code == 0, info
        Ptr = h.project(V, _dev(p.X)).cpu().numpy()
        Pte = h.project(V, _dev(p.Xtest)).cpu().numpy()
        return h.c2, lam.cpu().numpy(), V.cpu().numpy().T, info, Ptr, Pte


@pytest.mark.parametrize("name,tol,eig_tol,angle_tol", [
    ("d4096_k40", 1e-10, 1e-10, 1e-8),
    ("d16384_k100", 1e-8, 1e-6, 1e-6),
])
def test_mixed_precision_solver(eda, name, tol, eig_tol, angle_tol):
    c = synth.CONFIGS[name]
    p = synth.config_problem(name)
    c2, lam, V, info, Ptr, Pte = _run(eda, p, c["t"], c["b"], c["tau"], tol, eda.EDA_F32)
    assert info["refine_iters"] >= 1
    assert info["max_relres_true"] <= 10 * tol
    ref = O.eda(p.X, p.labels, p.k, c["t"], c2=c2, tier="projected")
    rel = np.abs(lam - ref["lam_t"]) / ref["lam_t"]
    assert rel.max() <= eig_tol, rel.max()
    assert O.sin_angle(ref["V"], V) <= angle_tol
    lab_g, _, _ = O.nn_classify(Ptr, p.labels, Pte)
    lab_o, _, _ = O.nn_classify(O.project(ref["V"], p.X), p.labels, O.project(ref["V"], p.Xtest))
    assert np.array_equal(lab_g, lab_o)


def test_mixed_matches_fp64_path_small(eda):
    p = synth.gaussian_clusters(d=500, k=6, n_per_class=[3, 4, 5, 2, 6, 3], seed=77, n_test_per_class=2)
    _, lam64, V64, _, _, _ = _run(eda, p, 5, 2, 8.0, 1e-10, eda.EDA_F64)
    _, lam32, V32, info, _, _ = _run(eda, p, 5, 2, 8.0, 1e-10, eda.EDA_F32)
    assert np.max(np.abs(lam32 - lam64) / lam64) <= 1e-10
    assert O.sin_angle(V64, V32) <= 1e-8
