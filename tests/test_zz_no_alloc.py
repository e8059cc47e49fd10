"""nlos_reduce_static, the allocation-free variant of nlos_reduce, against
nlos_reduce through the C ABI, on two calls in a row.

Some callers cannot allocate device memory at the point where they reduce a
cube (their memory is already reserved by another allocator, or their loop
cannot take the synchronisation of cudaMalloc/cudaFree); this entry point keeps
its scratch in a fixed device array instead. The second call uses fewer
transients than the first, so stale partials left in the shared array by the
first call must not leak into its result.

Collected last on purpose (file name): if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _ref(t, traces, B):
    from paper_2506_03747_gb300 import nlos
    en = torch.empty(traces, dtype=torch.float64, device="cuda")
    st = torch.empty(3, dtype=torch.float64, device="cuda")
    nlos.reduce(t, traces, B, en, st)
    torch.cuda.synchronize()
    return en.cpu().numpy(), st.cpu().numpy()


def _static(t, traces, B):
    from paper_2506_03747_gb300 import nlos
    en = torch.full((traces,), -1.0, dtype=torch.float64, device="cuda")
    st = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    nlos.reduce_static(t, traces, B, en, st)
    torch.cuda.synchronize()
    return en.cpu().numpy(), st.cpu().numpy()


def test_reduce_static_matches_reduce_on_two_calls():
    H.lib()
    rng = np.random.default_rng(2024)
    # first call: a large cube; second call: fewer transients, different bins
    for traces, B, scale in [(5000, 512, 1.0), (1234, 1023, 3.0)]:
        x = ((rng.random((traces, B)) ** 4) * scale).astype(np.float32)
        x[rng.random((traces, B)) < 0.3] = 0.0
        t = torch.from_numpy(x).cuda()
        e_ref, s_ref = _ref(t, traces, B)
        e_st, s_st = _static(t, traces, B)
        np.testing.assert_allclose(e_st, e_ref, rtol=1e-12, atol=0)
        assert s_st[0] == s_ref[0] == float(x.max())
        assert s_st[1] == pytest.approx(s_ref[1], rel=1e-12)
        assert s_st[2] == pytest.approx(s_ref[2], rel=1e-12)
        x64 = x.astype(np.float64)
        assert s_st[1] == pytest.approx(x64.sum(), rel=1e-12)


def test_reduce_static_rejects_more_transients_than_its_array():
    H.lib()
    from paper_2506_03747_gb300 import nlos
    t = torch.zeros((65537, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(nlos.NlosError) as ei:
        nlos.reduce_static(t, 65537, 4, None, None)
    assert ei.value.status == nlos.EINVAL


def test_reduce_static_optional_outputs_and_empty():
    """Either output may be omitted, and zero transients is a valid call (the
    statistics of an empty cube are zeros)."""
    H.lib()
    from paper_2506_03747_gb300 import nlos
    rng = np.random.default_rng(7)
    x = (rng.random((300, 256)) ** 3).astype(np.float32)
    t = torch.from_numpy(x).cuda()
    e_ref, s_ref = _ref(t, 300, 256)
    en = torch.full((300,), -1.0, dtype=torch.float64, device="cuda")
    nlos.reduce_static(t, 300, 256, en, None)
    st = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    nlos.reduce_static(t, 300, 256, None, st)
    torch.cuda.synchronize()
    np.testing.assert_allclose(en.cpu().numpy(), e_ref, rtol=1e-12, atol=0)
    np.testing.assert_allclose(st.cpu().numpy(), s_ref, rtol=1e-12, atol=0)
    st0 = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    nlos.reduce_static(t, 0, 256, None, st0)
    torch.cuda.synchronize()
    assert (st0.cpu().numpy() == 0.0).all()
