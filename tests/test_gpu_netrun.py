"""The messages of Pi_MultVerify^R on the GPU (the library's ledger) are exactly those the
communication model prices, for several D and R; the network-shaped run reports an R per network."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_09287_gb300 import mpc as M
    return M


def test_gpu_ledger_equals_the_model_and_a_best_R_exists(mpc):
    from paper_2411_09287_gb300 import netmodel as NM
    from paper_2411_09287_gb300 import netrun as NR
    D = 1000
    gpu = NR.measure(mpc, D, [0, 1, 3, 5, 8], reps=1)   # raises on a ledger mismatch
    for name, net in NM.NETWORKS.items():
        R, tot = NR.best_by_total(gpu, D, net)
        assert R in gpu and tot > 0
