"""The no-allocation exp-vector product against the regular entry point (GPU, through the C ABI).

eda_lowrank_exp_apply_noalloc serves callers that must not allocate device memory (a host
framework with a fixed memory budget, or a latency-critical loop); it keeps its temporaries in
a fixed array inside the library. Here it must reproduce eda_apply_exp on the same operator
within the tolerance the parity tests use for FP64 products (1e-12 relative), on two calls in
a row with different shapes, so that stale scratch contents from the first call cannot leak
into the second. This file is collected last so that a failure here stops a run only after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_1512_06500_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_eda_apply_exp_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_06500_gb300 import build_lib, eda
    build_lib.build()
    lib = eda.load()
    fn = lib.eda_lowrank_exp_apply_noalloc
    dev = "cuda:0"
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(4096, 40, 5, 8, 1), (777, 9, [2, 5, 3, 4, 6, 2, 3, 7, 1], 3, 2)]
    for d, k, nj, b, seed in cases:
        p = synth.gaussian_clusters(d=d, k=k, n_per_class=nj, seed=300 + seed)
        X = torch.from_numpy(p.X).to(dev)
        lab = torch.from_numpy(p.labels).to(dev)
        with eda.build(X, lab, p.k, eda.config(block_b=2, tau=10.0)) as h:
            f = h.factors()
            gen = torch.Generator(device="cpu").manual_seed(seed)
            Xb = torch.randn(b, d, generator=gen, dtype=torch.float64).to(dev)
            for op, H, K, alpha in ((eda.OP_SW, f["HW"], f["KW"], -0.5 * h.c2), (eda.OP_SB, f["HB"], f["KB"], h.c2)):
                Y_ref = h.apply_exp(op, Xb, alpha=alpha)
                Y = torch.full_like(Xb, float("nan"))
                m = H.shape[0]
                rc = fn(ctypes.c_void_p(H.data_ptr()), d, m, ctypes.c_void_p(K.data_ptr()),
                        ctypes.c_void_p(Xb.data_ptr()), ctypes.c_void_p(Y.data_ptr()), d, b, stream)
                assert rc == 0, eda.STATUS.get(rc, rc)
                torch.cuda.synchronize()
                err = (torch.linalg.norm(Y - Y_ref) / torch.linalg.norm(Y_ref)).item()
                assert err <= 1e-12, (d, op, err)
    # sizes beyond the fixed scratch are rejected before any device work
    big = torch.zeros(1, dtype=torch.float64, device=dev)
    ptr = ctypes.c_void_p(big.data_ptr())
    Yb = torch.zeros(1, dtype=torch.float64, device=dev)
    assert fn(ptr, 1, 2000, ptr, ptr, ctypes.c_void_p(Yb.data_ptr()), 1, 100, stream) == -1
