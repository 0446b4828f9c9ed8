"""The allocation-free Hamiltonian-constraint entry point (nr_hamiltonian_noalloc).

It serves callers that cannot call cudaMalloc -- a host framework that owns all
device memory, a caller without an nr_grid, a latency-critical loop -- by keeping
its scratch in one file-scope device array.  Checked here through the C ABI: two
calls in a row on different states agree with the grid-based nr_hamiltonian
within the tolerances of the other Hamiltonian tests (H 1e-12 relative, norms
1e-10) at both finite-difference orders, device free memory does not change across
calls, and grids beyond the
array's stated limit are rejected.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_00097_gb300 import binding as B  # noqa: E402
from paper_2505_00097_gb300 import build as BUILD  # noqa: E402
from paper_2505_00097_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

KO8 = [0.3] * 17 + [0.99] * 7
SPECS = [
    dict(W.sinh_spherical((37, 11, 6)), h_rmin=0.5, h_rmax=8.0),
    dict(W.sinh_cylindrical((33, 2, 70), rho_max=20.0, z_max=20.0), h_rmin=0.5, h_rmax=8.0),
    dict(W.sinh_spherical((37, 11, 6)), h_rmin=0.5, h_rmax=8.0, NG=5, ko_sigma=KO8),
    dict(W.sinh_cylindrical((33, 2, 70), rho_max=20.0, z_max=20.0), h_rmin=0.5, h_rmax=8.0, NG=5, ko_sigma=KO8),
    dict(W.spherical((21, 9, 8)), h_rmin=0.5, h_rmax=6.0),
]
IDS = ["sinhsph", "sinhcyl", "sinhsph-o8", "sinhcyl-o8", "spherical"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    BUILD.build()
    B.lib()


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("use_stream", [False, True], ids=["legacy-stream", "torch-stream"])
@pytest.mark.parametrize("spec", SPECS, ids=IDS)
def test_noalloc_matches_grid_hamiltonian_two_calls(spec, use_stream):
    g = B.Grid(spec)
    T = g.T
    # every input and output of both calls exists before the first call
    ys = [torch.from_numpy(W.random_state(g.n, seed=seed, smooth=True)).to("cuda:0") for seed in (101, 202)]
    H_ref = [torch.full((T,), float("nan"), dtype=torch.float64, device="cuda:0") for _ in ys]
    H_na = [torch.full((T,), float("nan"), dtype=torch.float64, device="cuda:0") for _ in ys]
    refs = [g.hamiltonian(y, h) for y, h in zip(ys, H_ref)]
    stream = torch.cuda.Stream() if use_stream else None
    handle = stream.cuda_stream if use_stream else None
    before, after = [], []
    for call, y in enumerate(ys):
        before.append(_free())
        l2, linf = B.hamiltonian_noalloc(spec, y, H_na[call], stream=handle)
        after.append(_free())
        a, b = H_na[call].cpu().numpy(), H_ref[call].cpu().numpy()
        assert np.all(np.isfinite(a))
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err <= 1e-12, (call, err)
        l2_ref, linf_ref = refs[call]
        assert l2 == pytest.approx(l2_ref, rel=1e-10)
        assert linf == pytest.approx(linf_ref, rel=1e-10)
        # norms only, no H output
        before.append(_free())
        l2b, linfb = B.hamiltonian_noalloc(spec, y, stream=handle)
        after.append(_free())
        assert l2b == pytest.approx(l2_ref, rel=1e-10) and linfb == pytest.approx(linf_ref, rel=1e-10)
    # device free memory is the same on either side of every call after the first (which sets up
    # the device address of the scratch array)
    assert before[1:] == after[1:], (before, after)
    g.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    """n0 = 20006: the per-axis arrays need 4*20006 + 4*8 + 2*8 = 80,072 doubles > 59,360.  The
    state buffer handed over is a real device buffer of the grid's full size, so the call reads
    nothing out of bounds even if the size check were missing."""
    spec = W.sinh_spherical((20000, 2, 2))
    T = (20000 + 6) * 8 * 8
    y = torch.zeros(24 * T, dtype=torch.float64, device="cuda:0")
    with pytest.raises(B.NrError) as ei:
        B.hamiltonian_noalloc(spec, y)
    assert ei.value.code == 1 and "static scratch" in str(ei.value)
