"""colapm_power_noalloc against colapm_power, through the C ABI.

colapm_power_noalloc serves callers that cannot allocate device memory (code inside another
framework's memory budget or allocator, or loops where cudaMalloc's implicit synchronisation
is not allowed): its working memory is one fixed device array inside the library. It must
give what the context-based colapm_power gives for the same positions, on consecutive calls
(the shared array keeps the previous call's contents, which each call must clear).
This file is collected last so that a failure here stops a -x run only after every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    from paper_1506_03737_gb300 import colapm
    return colapm


@pytest.mark.parametrize("np_,nm,nbins", [(32, 64, 100), (64, 128, 37)])
def test_noalloc_power_matches_context_power(C, np_, nm, nbins):
    import torch
    box = 256.0
    ctx = C.colapm_create(C.default_params(np=np_, nm=nm, box=box, seed=21))
    try:
        C.colapm_make_ics(ctx)
        C.colapm_step(ctx, 3)
        n = np_ ** 3
        cell = np.empty((n, 3), np.int32)
        off = np.empty((n, 3), np.float32)
        C.colapm_get_state(ctx, cell, off, None)
        k_ref, p_ref, n_ref = C.colapm_power(ctx, nbins)
    finally:
        C.colapm_destroy(ctx)
    cell_d = torch.from_numpy(cell).cuda()
    off_d = torch.from_numpy(off).cuda()
    torch.cuda.synchronize()
    ok = n_ref > 0
    for _ in range(2):                       # two calls in a row share the fixed scratch array
        k, p, cnt = C.colapm_power_noalloc(cell_d, off_d, n, nm, box, nbins)
        assert np.array_equal(cnt, n_ref)
        assert np.max(np.abs(p[ok] / p_ref[ok] - 1)) < 1e-4
        assert np.max(np.abs(k[ok] / k_ref[ok] - 1)) < 1e-12


def test_noalloc_rejects_oversize_and_host_inputs(C):
    import torch
    cell = torch.zeros((8, 3), dtype=torch.int32, device="cuda")
    off = torch.zeros((8, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(C.ColapmError) as e:
        C.colapm_power_noalloc(cell, off, 8, 256, 100.0, 10)        # nm above the maximum
    assert e.value.code == -1
    with pytest.raises(C.ColapmError) as e:
        C.colapm_power_noalloc(cell, off, 8, 64, 100.0, 1000)       # too many bins
    assert e.value.code == -1
    with pytest.raises(C.ColapmError) as e:
        C.colapm_power_noalloc(cell.cpu().numpy(), off.cpu().numpy(), 8, 64, 100.0, 10)   # host inputs
    assert e.value.code == -1


def test_noalloc_rejects_arrays_on_another_gpu(C):
    # The call runs on the current device; positions held by another GPU are refused on the host,
    # before anything is queued.
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second GPU")
    cell = torch.zeros((8, 3), dtype=torch.int32, device="cuda:1")
    off = torch.zeros((8, 3), dtype=torch.float32, device="cuda:1")
    torch.cuda.set_device(0)
    with pytest.raises(C.ColapmError) as e:
        C.colapm_power_noalloc(cell, off, 8, 64, 100.0, 10)
    assert e.value.code == -1


def test_noalloc_reports_a_full_cell(C):
    # 2^18 particles on one node put 2^63 into one cell of the fixed-point mesh: an overflow the
    # deposit itself reports, whatever the particle count.
    import torch
    n = 1 << 18
    cell = torch.zeros((n, 3), dtype=torch.int32, device="cuda")
    off = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(C.ColapmError) as e:
        C.colapm_power_noalloc(cell, off, n, 16, 100.0, 10)
    assert e.value.code == -4
    # the next call clears the shared array and succeeds
    k, p, cnt = C.colapm_power_noalloc(cell[:8], off[:8], 8, 16, 100.0, 10)
    assert cnt.sum() > 0
