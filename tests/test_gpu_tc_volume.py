"""The volume term of the Q3 KPP problem on the tensor cores against the CUDA cores
(dgw_selftest_tc_volume): both against an FP64 evaluation written out with NumPy, and the
time of each on the 1024^2 workload's cell count (recorded, not a pass condition)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2309_12019_gb300 import dgw
from paper_2309_12019_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dgw.load()


def volume_fp64(U):
    """acc_(i+4j) = sum_q w_qx w_qy [P_i'(x) P_j(y) sin u + P_i(x) P_j'(y) cos u] at the 5 x 5
    Gauss points, u = sum c_(i+4j) P_i(x) P_j(y) (Eq. weak2 for F = (sin u, cos u))."""
    g, w = np.polynomial.legendre.leggauss(5)
    P = np.array([np.polynomial.legendre.legval(g, np.eye(4)[i]) for i in range(4)])          # [i][q]
    D = np.array([np.polynomial.legendre.legval(g, np.polynomial.legendre.legder(np.eye(4)[i])) for i in range(4)])
    C = U.reshape(4, 4, -1)                                   # [j][i][e]
    u = np.einsum("ia,jb,jie->eab", P, P, C)                  # [e][qx][qy]
    fx, fy = np.sin(u), np.cos(u)
    acc = (np.einsum("a,b,ia,jb,eab->jie", w, w, D, P, fx) + np.einsum("a,b,ia,jb,eab->jie", w, w, P, D, fy))
    return acc.reshape(16, -1)


def test_tc_volume_matches_fp64_and_cuda_cores():
    ntiles = 64
    U = I.random_state(2, 3, ntiles * 128, seed=5, smooth=True, scale=3.0, offset=5.0)
    ref = volume_fp64(U)
    Ud = torch.tensor(U, dtype=torch.float32, device="cuda")
    scale = np.max(np.abs(ref))
    for variant in (0, 1):
        out = torch.empty_like(Ud)
        dgw.selftest_tc_volume(Ud, out, variant)
        got = out.double().cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-5 * scale, (variant, np.max(np.abs(got - ref)) / scale)


def test_tc_volume_timing():
    """Both variants on 8192 tiles (1,048,576 cells: the KPP workload's count)."""
    ntiles = 8192
    Ud = torch.rand((16, ntiles * 128), dtype=torch.float32, device="cuda") * 3.0 + 5.0
    out = torch.empty_like(Ud)
    t = {}
    for variant in (0, 1):
        dgw.selftest_tc_volume(Ud, out, variant)          # warm-up
        t[variant] = min(dgw.selftest_tc_volume(Ud, out, variant) for _ in range(5))
    print(f"volume term of 1,048,576 Q3 cells: CUDA cores {1e3 * t[0]:.1f} us, tensor cores {1e3 * t[1]:.1f} us")
    assert t[0] > 0 and t[1] > 0
