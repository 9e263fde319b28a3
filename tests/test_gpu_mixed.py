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
    # returns the library's c^2 only to check it against the oracle's own (no oracle input comes from it)
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
    ref = O.eda(p.X, p.labels, p.k, c["t"], tau=c["tau"], tier="projected")
    assert abs(c2 - ref["c2"]) <= 1e-13 * ref["c2"]
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


def _near_midpoint_ulp(v, rel):
    """bf16 ulp of each entry of v whose FP64 value lies within rel |v| of a bf16 rounding midpoint (where an
    FP32 accumulation of the same value may round to the other neighbour), else 0."""
    m, e = np.frexp(v)
    ulp = np.ldexp(1.0, e - 8)                         # 8 significant bits
    f = v / ulp
    dist = np.abs(f - np.floor(f) - 0.5) * ulp
    return np.where(dist <= rel * np.abs(v), ulp, 0.0)


@pytest.mark.parametrize("d,k,nj,b", [(4096, 40, 5, 8), (1000, 9, [2, 5, 3, 4, 6, 2, 3, 7, 1], 16), (2048, 20, 7, 32),
                                      (777, 5, 3, 40)])
def test_tc_exp_apply_matches_bf16_reference(eda, d, k, nj, b):
    # The tensor-core product is X + bf16(H K) (bf16(H)^T X): H and the precomputed d x m product H K
    # are stored in bf16, X and P = H^T X enter as hi + lo bf16 pairs, accumulation is FP32. The
    # reference takes H from the oracle's scatter factors and K = alpha phi(alpha G) from the oracle's
    # Gram and scale, applies the same bf16 roundings in FP64 and is compared element by element. Allowed:
    # 1e-4 of the column's largest entry (hi + lo rounding of X and P, 2^-17, and FP32 accumulation), plus,
    # for each entry of H K whose FP64 value sits within 1e-4 of a bf16 rounding midpoint (there the
    # kernel's FP32-accumulated H K may round to the other neighbour), one bf16 ulp of it times |P|. Any
    # operand or layout mistake (a transposed core matrix, a wrong swizzle, a wrong K step, a lost tile
    # edge at a ragged d) exceeds this by orders of magnitude.
    p = synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=500 + d)
    f = O.scatter_factors(p.X, p.labels, p.k)
    GW, GB = O.gram(f["HW"]), O.gram(f["HB"])
    c2 = O.scale_c2(np.linalg.eigvalsh(GW)[-1], np.linalg.eigvalsh(GB)[-1], 10.0)
    cfg = eda.config(prec=eda.EDA_BF16, block_b=min(b, 16), tau=10.0, tc_fused=-1)   # the four-launch sweeps
    with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
        assert abs(h.c2 - c2) <= 1e-13 * c2
        rng = np.random.default_rng(d + b)
        Xb = rng.standard_normal((b, d)).astype(np.float32)
        # the library's alpha selects its stored bf16 operators
        for op, H, G, a_lib, a_ref in ((eda.OP_SW, f["HW"], GW, -0.5 * h.c2, -0.5 * c2),
                                       (eda.OP_SB, f["HB"], GB, h.c2, c2)):
            Y = h.apply_exp(op, _dev(Xb), alpha=a_lib).cpu().numpy().astype(np.float64).T   # d x b
            K = O.phi_operator(G, a_ref)
            Hb = _bf16_round(H.T)                      # (m, d): rows are the columns of H
            HK = Hb.T @ K                              # (d, m), FP64
            HKb = _bf16_round(HK)
            X64 = Xb.astype(np.float64).T              # d x b
            P = Hb @ X64                               # m x b
            ref = X64 + HKb @ P
            tol = 1e-4 * np.abs(ref).max(axis=0)[None, :] + _near_midpoint_ulp(HK, 1e-4) @ np.abs(P)
            err = np.abs(Y - ref)
            assert np.all(err <= tol), (op, float((err / tol).max()))
            # against the exact FP64 operator: the bf16 rounding of H and H K (2^-9) sets the scale
            exact = O.lowrank_exp_apply(H, a_ref, X64)
            scale = np.abs(X64) + np.abs(HK) @ np.abs(P)
            assert np.all(np.abs(Y - exact) <= 2e-2 * scale.max(axis=0)[None, :]), op


@pytest.mark.parametrize("d,k,nj,b", [(4096, 40, 5, 8), (1000, 9, [2, 5, 3, 4, 6, 2, 3, 7, 1], 16), (2048, 20, 7, 20),
                                      (777, 5, 3, 40), (16384, 100, 7, 16), (300, 150, 2, 32), (100, 6, 4, 5)])
def test_tc_fused_exp_apply_matches_bf16_reference(eda, d, k, nj, b):
    # The one-pass product is X + sigma bf16(B) (bf16(B)^T X) with B = H R^T, sigma K = R^T R (Cholesky of the
    # definite K = alpha phi(alpha G), sigma = sign(alpha)): one d x m bf16 matrix serves both sweeps and stays
    # in shared memory. The reference forms B from the oracle's H, Gram and scale in FP64, rounds it to bf16
    # as the library does, and applies it in FP64; allowed: 1e-4 of the column's largest entry (hi + lo
    # rounding of X and P, FP32 accumulation) plus one bf16 ulp of each entry of B within 1e-4 of a rounding
    # midpoint times |P|. Covers one to six 128-column bands, ragged d, a single CTA (d = 100), b of 5 to 40
    # (two launches); the
    # in-place form (Y = X) runs inside the bf16 solver's M-apply chain (test_bf16_tensor_core_solver).
    p = synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=900 + d)
    f = O.scatter_factors(p.X, p.labels, p.k)
    GW, GB = O.gram(f["HW"]), O.gram(f["HB"])
    c2 = O.scale_c2(np.linalg.eigvalsh(GW)[-1], np.linalg.eigvalsh(GB)[-1], 10.0)
    cfg = eda.config(prec=eda.EDA_BF16, block_b=min(b, 16), tau=10.0)
    with eda.build(_dev(p.X), _dev(p.labels), p.k, cfg) as h:
        assert abs(h.c2 - c2) <= 1e-13 * c2
        rng = np.random.default_rng(d + b)
        Xb = rng.standard_normal((b, d)).astype(np.float32)
        for op, H, G, a_lib, a_ref in ((eda.OP_SW, f["HW"], GW, -0.5 * h.c2, -0.5 * c2),
                                       (eda.OP_SB, f["HB"], GB, h.c2, c2)):
            Y = h.apply_exp(op, _dev(Xb), alpha=a_lib).cpu().numpy().astype(np.float64).T
            K = O.phi_operator(G, a_ref)
            sigma = 1.0 if a_ref > 0 else -1.0
            L = np.linalg.cholesky(sigma * K)          # sigma K = L L^T, B = H L
            B = H @ L
            Bb = _bf16_round(B)
            X64 = Xb.astype(np.float64).T
            P = Bb.T @ X64
            ref = X64 + sigma * (Bb @ P)
            tol = 1e-4 * np.abs(ref).max(axis=0)[None, :] + _near_midpoint_ulp(B, 1e-4) @ np.abs(P)
            err = np.abs(Y - ref)
            assert np.all(err <= tol), (op, float((err / tol).max()))
            exact = O.lowrank_exp_apply(H, a_ref, X64)
            scale = np.abs(X64) + np.abs(B) @ np.abs(P)
            assert np.all(np.abs(Y - exact) <= 2e-2 * scale.max(axis=0)[None, :]), op


@pytest.mark.parametrize("name,tol,eig_tol", [("d4096_k40", 1e-8, 1e-6), ("d16384_k100", 1e-8, 1e-6)])
def test_bf16_tensor_core_solver(eda, name, tol, eig_tol):
    c = synth.CONFIGS[name]
    p = synth.config_problem(name)
    c2, lam, V, info, Ptr, Pte = _run(eda, p, c["t"], c["b"], c["tau"], tol, eda.EDA_BF16)
    assert info["refine_iters"] >= 1
    assert info["max_relres_true"] <= 10 * tol
    ref = O.eda(p.X, p.labels, p.k, c["t"], tau=c["tau"], tier="projected")
    assert abs(c2 - ref["c2"]) <= 1e-13 * ref["c2"]
    rel = np.abs(lam - ref["lam_t"]) / ref["lam_t"]
    assert rel.max() <= eig_tol, rel.max()
    lab_g, _, _ = O.nn_classify(Ptr, p.labels, Pte)
    lab_o, _, _ = O.nn_classify(O.project(ref["V"], p.X), p.labels, O.project(ref["V"], p.Xtest))
    assert np.array_equal(lab_g, lab_o)
