"""The integer-pipe exact binary64 arithmetic (used for d-bar on the GPU) equals
the hardware FP64 unit bit for bit: x - y, m * m, x + y, G in 2D/3D and d-bar in
2D/3D against a plain bisection over the hardware G (through the C ABI)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_05694_gb300 as eik  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2103_05694_gb300 import build
    build.build()
    eik.load_library()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_exact_arithmetic_matches_fp64_unit(seed):
    res = eik.eik_selftest(n=1 << 22, seed=seed)
    assert res["trials"] == 1 << 22
    for k in eik.SELFTEST_CHECKS:
        assert res[k] == 0, (k, res)
