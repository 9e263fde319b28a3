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


# ----------------------------------------------------------------- bf16 tensor-core exp-apply

def _bf16_round(a):
    """float64 -> float32 -> bfloat16 (round to nearest even) -> float64, as the kernels convert H."""
    t = torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.to(torch.float64).numpy()


@pytest.mark.parametrize("d,k,nj,b", [(4096, 40, 5, 8), (1000, 9, [2, 5, 3, 4, 6, 2, 3, 7, 1], 16), (2048, 20, 7, 32),
                                      (777, 5, 3, 40)])
def test_tc_exp_apply_matches_bf16_reference(eda, d, k, nj, b):
    # The tensor-core product is X + bf16(H K) (bf16(H)^T X): H and the precomputed d x m product H K
    # are stored in bf16, X and P = H^T X enter as hi + lo bf16 pairs, accumulation is FP32. Against an
    # FP64 evaluation of that expression the error is the hi + lo rounding (2^-17 relative), FP32
    # accumulation, and the rare entries of H K whose FP32 and FP64 values round to different bf16
    # neighbours, so 1e-4 relative is a sharp bound that any operand or layout mistake (a transposed
    # core matrix, a wrong swizzle, a wrong K step) violates by orders of magnitude.
    p = synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=500 + d)
    cfg = eda.config(prec=eda.EDA_BF16, block_b=min(b, 16), tau=10.0)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
        f = h.factors()
        rng = np.random.default_rng(d + b)
        Xb = rng.standard_normal((b, d)).astype(np.float32)
        for op, H, K, alpha in ((eda.OP_SW, f["HW"], f["KW"], -0.5 * h.c2), (eda.OP_SB, f["HB"], f["KB"], h.c2)):
            Y = h.apply_exp(op, _dev(Xb), alpha=alpha).cpu().numpy().astype(np.float64)
            Hn = H.cpu().numpy()                       # (m, d): rows are the columns of H
            Hb = _bf16_round(Hn)
            Kn = K.cpu().numpy()
            HKb = _bf16_round(Hb.T @ Kn)               # (d, m)
            X64 = Xb.astype(np.float64)
            ref = X64 + (HKb @ (Hb @ X64.T)).T
            err = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
            assert err <= 1e-4, (op, err)
            # and against the exact FP64 operator: the bf16 rounding of H and H K (2^-9) sets the scale
            exact = X64 + ((Hn.T @ (Kn @ (Hn @ X64.T))).T)
            assert np.linalg.norm(Y - exact) / np.linalg.norm(exact) <= 2e-2


@pytest.mark.parametrize("name,tol,eig_tol", [("d4096_k40", 1e-8, 1e-6), ("d16384_k100", 1e-8, 1e-6)])
def test_bf16_tensor_core_solver(eda, name, tol, eig_tol):
    c = synth.CONFIGS[name]
    p = synth.config_problem(name)
    c2, lam, V, info, Ptr, Pte = _run(eda, p, c["t"], c["b"], c["tau"], tol, eda.EDA_BF16)
    assert info["refine_iters"] >= 1
    assert info["max_relres_true"] <= 10 * tol
    ref = O.eda(p.X, p.labels, p.k, c["t"], c2=c2, tier="projected")
    rel = np.abs(lam - ref["lam_t"]) / ref["lam_t"]
    assert rel.max() <= eig_tol, rel.max()
    lab_g, _, _ = O.nn_classify(Ptr, p.labels, Pte)
    lab_o, _, _ = O.nn_classify(O.project(ref["V"], p.X), p.labels, O.project(ref["V"], p.Xtest))
    assert np.array_equal(lab_g, lab_o)
