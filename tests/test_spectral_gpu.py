"""rd_spectral_radius: the Collatz-Wielandt bracket of rho(X) (Theorem 1's convergence condition)
from power iteration on the GPU against the oracle's dense eigenvalues."""
import numpy as np
import pytest

import oracle
from paper_2308_07403_gb300 import graphs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_07403_gb300 import build
    from paper_2308_07403_gb300 import rd as _rd

    build.build()
    _rd.load()
    return _rd


CASES = {
    "er300": lambda: (graphs.er(300, 0.03, 3), None, None),
    "ws500": lambda: (graphs.ws(500, 10, 0.1, 4), None, None),
    "grid400": lambda: (graphs.grid4(400, 20), None, None),
    "cycle257": lambda: (graphs.directed_cycle(257), None, None),
    "king_weighted": lambda: graphs.workload_weighted(12, 16) + (None,),
}


@pytest.mark.parametrize("name", list(CASES))
def test_bracket_contains_rho_and_closes(rd, name):
    A, W, g = CASES[name]()[:3]
    if g is None:
        g = graphs.gamma_frac(A, 0.9)
    rho = oracle.spectral_radius(A, g, W)
    with rd.Handle(A, g, W=W) as h:
        lo1, hi1 = h.spectral_radius(1)
        lo, hi = h.spectral_radius(3000)
    # one step from x = 1: the largest ratio is the largest column sum of X
    assert lo1 <= rho * (1 + 1e-12) and rho <= hi1 * (1 + 1e-12)
    assert lo <= rho * (1 + 1e-12) and rho <= hi * (1 + 1e-12), (lo, rho, hi)
    assert hi - lo <= 1e-6 * rho, (lo, rho, hi)   # strongly connected: the bracket closes
    assert hi < 1.0                                  # the gain check implies convergence


def test_acyclic_graph_has_zero_radius(rd):
    """A directed path is nilpotent: rho = 0 lies in the bracket and its lower end is 0."""
    A = graphs.directed_path(200)
    g = 0.5
    with rd.Handle(A, g) as h:
        lo, hi = h.spectral_radius(50)
    assert lo == 0.0 and 0.0 <= hi < 1.0


def test_bad_arguments(rd):
    A = graphs.er(64, 0.1, 1)
    with rd.Handle(A, graphs.gamma_frac(A, 0.5)) as h:
        with pytest.raises(rd.RDError):
            h.spectral_radius(0)
