"""The Python binding fails loudly on the host: no CPU fallback, no silent copies.

No GPU needed: every check below raises before a CUDA call is made.
"""
import pytest

torch = pytest.importorskip("torch")

from paper_1808_04580_gb300 import nfl


def test_plan_rejects_host_nodes():
    with pytest.raises(TypeError):
        nfl.Plan(torch.zeros((10, 3), dtype=torch.float64), 0.5, 16, 3)


def test_plan_rejects_other_dtypes():
    with pytest.raises(TypeError):
        nfl.Plan(torch.zeros((10, 3), dtype=torch.float32), 0.5, 16, 3)


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(nfl, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(nfl, "_LIB", None)
    with pytest.raises(RuntimeError):
        nfl.library()


def test_precisions_and_kernels_are_the_header_values():
    assert nfl.PRECISIONS == {"fp64": 0, "fp32": 1, "fp32c": 2, "bf16w": 3}
    assert nfl.KERNELS == {"gaussian": 0, "laplacian_rbf": 1, "multiquadric": 2, "inverse_multiquadric": 3,
                           "gaussian_dsigma": 4}


def test_apply_host_rejects_device_or_wrong_dtype_input():
    class Fake:        # a plan object without a library handle: the checks come first
        n = 4
    with pytest.raises(TypeError):
        nfl.Plan.apply_host(Fake(), torch.zeros(4, dtype=torch.float32))
