"""dvm_moments_noalloc: the moment and flow-rate reduction of dvm_moments without any device
allocation (its scratch is a fixed array inside the library), for callers that cannot allocate during
a call.  Checked through the C ABI against dvm_moments on the same input, on two calls in a row (the
shared scratch keeps the previous call's contents, so the second call checks that nothing leaks).
Kept in its own file, collected last, so a failure here leaves every other test already run."""
import numpy as np
import pytest

from paper_1704_03126_gb300 import build as dvm_build
from paper_1704_03126_gb300 import dvm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built_library():
    dvm_build.build()
    return dvm.lib()


def _run(h, mask, quad, dA, noalloc):
    import torch

    dev = torch.device("cuda")
    th = torch.from_numpy(np.ascontiguousarray(h)).to(dev)
    tm = torch.from_numpy(np.ascontiguousarray(mask.astype(np.uint8))).to(dev)
    mom = torch.full((h.shape[1], 4), float("nan"), dtype=torch.float64, device=dev)
    q = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    dvm.moments(th.data_ptr(), h.shape[1], quad, mom.data_ptr(), q.data_ptr(), dA, mask_ptr=tm.data_ptr(),
                stream=stream.cuda_stream, noalloc=noalloc)
    stream.synchronize()
    return mom.cpu().numpy(), float(q.cpu().item())


@pytest.mark.parametrize("ncell,quad", [(257 * 1031 + 17, ("nc", 6, 4.0)), (53, ("gh", 8, 0.0))])
def test_noalloc_matches_allocating_entry_point_twice(ncell, quad):
    rng = np.random.default_rng(2024)
    K = quad[1] ** 2
    dA = 1.0 / 4096.0
    for call in range(2):
        h = rng.standard_normal((K, ncell)) * (1.0 + call)
        mask = (rng.random(ncell) < 0.15).astype(np.uint8)
        mom_ref, q_ref = _run(h, mask, quad, dA, noalloc=False)
        mom, q = _run(h, mask, quad, dA, noalloc=True)
        scale = max(1.0, np.abs(mom_ref).max())
        assert np.abs(mom - mom_ref).max() < 1e-12 * scale
        assert abs(q - q_ref) < 1e-12 * max(1.0, abs(q_ref))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    with pytest.raises(dvm.DvmError) as ei:
        dvm.moments(1, 16_777_217, ("gh", 4, 0.0), 1, 1, 1.0, noalloc=True)
    assert ei.value.status == dvm.DVM_EINVAL
    assert "exceeds this call's maximum" in str(ei.value)
