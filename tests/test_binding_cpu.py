"""The Python binding refuses what the library cannot run before it reaches the library: there
is no CPU path, so CPU tensors, unsupported dtypes, mismatched shapes and unknown host-transfer
modes are errors (runs without a GPU; no compute calls)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2108_11560_gb300 import kv  # noqa: E402


def _cpu(n=4, dtype=None):
    return torch.linspace(0.5, 2.0, n, dtype=dtype or torch.float64)


@pytest.mark.parametrize("fn", [kv.kv_log, kv.kv_log_dv, kv.kv_log_dx, kv.kv_fwd_bwd])
def test_cpu_tensors_are_refused(fn):
    with pytest.raises(ValueError, match="CUDA"):
        fn(_cpu(), _cpu())


def test_extended_call_and_autograd_refuse_cpu_tensors():
    with pytest.raises(ValueError, match="CUDA"):
        kv.kv_fwd_bwd_ex(_cpu(dtype=torch.float32), _cpu(dtype=torch.float32), bracket="f32")
    with pytest.raises(ValueError, match="CUDA"):
        kv.log_besselk(_cpu().requires_grad_(), _cpu())
    with pytest.raises(ValueError, match="CUDA"):
        kv.kv_bracket(_cpu(), _cpu())


def test_non_tensor_inputs_are_refused():
    with pytest.raises(TypeError):
        kv.kv_fwd_bwd(np.ones(4), np.ones(4))


def test_host_call_argument_checks():
    a = np.linspace(0.5, 2.0, 8)
    with pytest.raises(TypeError, match="float64 or float32"):
        kv.kv_fwd_bwd_host(a.astype(np.float16), a.astype(np.float16))
    with pytest.raises(ValueError, match="same dtype and shape"):
        kv.kv_fwd_bwd_host(a, a[:4])
    with pytest.raises(ValueError, match="same dtype and shape"):
        kv.kv_fwd_bwd_host(a, a.astype(np.float32))
    with pytest.raises(ValueError, match="transfer"):
        kv.kv_fwd_bwd_host(a, a, transfer="zero-copy")
    assert set(kv.HOST_TRANSFER) == {"auto", "staged", "direct"}
