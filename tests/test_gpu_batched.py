"""Batched solves (eda_solve_batched) against the oracle, problem by problem.

The batch runs the single-problem path for every problem on several host workers and streams; the
results must be what the oracle gives for each problem alone: eigenvalues to 1e-10 relative and
principal angles to 1e-8 for the FP64 path, 1e-6 for the bf16 tensor-core path, identical 1-NN labels.
The 64-problem workload of uneven d, k, n_j is checked problem by problem, in FP64, in the tensor-core
FP64 mode and with bf16 sweeps.
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


def _check(eda, p, res, c2, eig_tol, angle_tol, ref=None):
    t = res["lam"].shape[0]
    if ref is None:
        ref = O.eda(p.X, p.labels, p.k, t, c2=c2, tier="projected")
    lam = res["lam"].cpu().numpy()
    rel = np.abs(lam - ref["lam_t"]) / ref["lam_t"]
    assert rel.max() <= eig_tol, (p.name, rel.max())
    V = res["V"].cpu().numpy().T
    assert O.sin_angle(ref["V"], V) <= angle_tol, p.name
    Ptr, Pte = O.project(V, p.X), O.project(V, p.Xtest)
    lab_g, _, _ = O.nn_classify(Ptr, p.labels, Pte)
    lab_o, _, _ = O.nn_classify(O.project(ref["V"], p.X), p.labels, O.project(ref["V"], p.Xtest))
    assert np.array_equal(lab_g, lab_o), p.name


def _c2(p, tau):
    f = O.scatter_factors(p.X, p.labels, p.k)
    lw = float(np.linalg.eigvalsh(O.gram(f["HW"]))[-1])
    lb = float(np.linalg.eigvalsh(O.gram(f["HB"]))[-1])
    return O.scale_c2(lw, lb, tau)


def _problems(specs):
    out = []
    for i, (d, k, nj) in enumerate(specs):
        out.append(synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=900 + i, n_test_per_class=2,
                                           name=f"small{i}"))
    return out


def test_batched_fp64_uneven_matches_oracle(eda):
    specs = [(300, 4, [3, 2, 4, 3]), (1000, 9, 3), (512, 3, [5, 2, 7]), (777, 6, [2, 3, 4, 2, 3, 5]),
             (256, 5, 4), (1024, 12, [3] * 6 + [4] * 6)]
    ps = _problems(specs)
    tau = 10.0
    cfg = eda.config(prec=eda.EDA_F64, block_b=0, tau=tau)        # block size tuned per shape
    probs = [dict(X=_dev(p.X), labels=_dev(p.labels), k=p.k, t=p.k - 1, tol=1e-12) for p in ps]
    res, code = eda.solve_batched(probs, cfg, workers=3)
    assert code == 0, [r["status"] for r in res]
    for p, r in zip(ps, res):
        assert r["status"] == 0
        assert r["info"]["converged"] == p.k - 1
        _check(eda, p, r, _c2(p, tau), 1e-10, 1e-8)


def test_batched_bf16_matches_oracle(eda):
    ps = _problems([(2048, 10, 4), (1500, 7, [3, 4, 5, 3, 2, 6, 3]), (4096, 20, 3)])
    tau = 10.0
    cfg = eda.config(prec=eda.EDA_BF16, block_b=8, tau=tau)
    probs = [dict(X=_dev(p.X), labels=_dev(p.labels), k=p.k, t=p.k - 1, tol=1e-8) for p in ps]
    res, code = eda.solve_batched(probs, cfg, workers=2)
    assert code == 0, [r["status"] for r in res]
    for p, r in zip(ps, res):
        _check(eda, p, r, _c2(p, tau), 1e-6, 1e-5)


@pytest.fixture(scope="module")
def batch64():
    # the 64-problem workload and the oracle's answer for every problem (computed once for both precisions)
    ps = synth.batched_problems(64)
    tau = synth.BATCHED["tau"]
    refs = []
    for p in ps:
        c2 = _c2(p, tau)
        refs.append((c2, O.eda(p.X, p.labels, p.k, p.k - 1, c2=c2, tier="projected")))
    return ps, tau, refs


@pytest.mark.parametrize("prec_name", ["f64", "tc", "bf16"])
def test_batched_64_problem_workload_all(eda, batch64, prec_name):
    # bf16: the batch's own precision (bf16 sweeps on the tensor cores, FP64 small steps and refinement) to
    # tol 1e-8, held to the mixed-precision bars (eigenvalues 1e-6 relative, identical 1-NN labels)
    ps, tau, refs = batch64
    prec = {"f64": eda.EDA_F64, "tc": eda.EDA_F64_TC, "bf16": eda.EDA_BF16}[prec_name]
    tol = 1e-8 if prec_name == "bf16" else 1e-10
    cfg = eda.config(prec=prec, block_b=0, tau=tau)
    probs = [dict(X=_dev(p.X), labels=_dev(p.labels), k=p.k, t=p.k - 1, tol=tol) for p in ps]
    res, code = eda.solve_batched(probs, cfg, workers=16)
    assert code == 0, [r["status"] for r in res]
    assert all(r["status"] == 0 for r in res)
    # every problem against the oracle, one by one
    for p, r, (c2, ref) in zip(ps, res, refs):
        assert abs(r["info"]["c2"] - c2) <= 1e-13 * c2, p.name
        if prec_name == "bf16":
            _check(eda, p, r, c2, 1e-6, 1e-5, ref=ref)
        else:
            _check(eda, p, r, c2, 1e-9, 1e-7, ref=ref)
