"""A bounded device wait that runs out is reported as EDA_ERR_TIMEOUT, and the context stays usable.

The symmetric eigensolver of matrices above 512 rows runs as one cooperative grid whose CTAs meet at a
software grid barrier; every wait there polls at most eda_config.wait_limit times, then records a timeout
in the handle's status word and lets the kernel run to its end (no index depends on the data, so stale
values cannot send an access out of bounds). The host reads the status before it uses any result. Here a
limit of one poll makes the waits run out; nothing faults, traps or hangs.
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


def test_grid_barrier_timeout_is_reported_and_context_survives(eda):
    # n = 600 > 512: the build's eigensolve of G_W (n > 256 takes the eigenpair route) is the cooperative one
    p = synth.gaussian_clusters(d=1024, k=60, n_per_class=10, seed=77)
    X, lab = _dev(p.X), _dev(p.labels)
    with pytest.raises(eda.EdaError) as e:
        eda.build(X, lab, p.k, eda.config(tau=10.0, wait_limit=1))
    assert e.value.code == -6, e.value
    # the same problem with the default limit: the device and the library are still usable
    f = O.scatter_factors(p.X, p.labels, p.k)
    lw = float(np.linalg.eigvalsh(O.gram(f["HW"]))[-1])
    lb = float(np.linalg.eigvalsh(O.gram(f["HB"]))[-1])
    c2 = O.scale_c2(lw, lb, 10.0)
    with eda.build(X, lab, p.k, eda.config(tau=10.0)) as h:
        assert abs(h.c2 - c2) <= 1e-13 * c2
        V, lam, _, info, code = h.solve(p.k - 1, 1e-8)
        assert code == 0, info
    torch.cuda.synchronize()
