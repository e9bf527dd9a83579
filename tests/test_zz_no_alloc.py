"""The allocation-free inverse entry point, through the C ABI.

bt_zinv_batched_noalloc serves callers that cannot allocate device memory when they need an
inverse (code inside its own pool allocator, or with every free byte already given to an
arena): its scratch is a fixed array inside the library.  This file is collected last so that a
failure here never hides the other GPU tests; it also passes alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _inputs(rng, n, batch):
    A = rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))
    A += 2.0 * np.eye(n)
    return A


@pytest.mark.parametrize("n,batch", [(416, 8), (130, 5), (40, 3)])
def test_noalloc_matches_allocating_entry_point_on_two_calls(n, batch):
    import torch
    import paper_2508_19138_gb300 as pkg
    rng = np.random.default_rng(n + batch)
    for call in range(2):  # two calls in a row share the scratch array
        A = _inputs(rng, n, batch)
        ref = torch.from_numpy(A).cuda()
        got = ref.clone()
        info_ref = torch.zeros(batch, dtype=torch.int32, device="cuda")
        info_got = torch.full((batch,), 7, dtype=torch.int32, device="cuda")
        info_got.zero_()
        pkg.bt_zinv_batched(n, ref, n * n, batch, info_ref)
        pkg.bt_zinv_batched_noalloc(n, got, n * n, batch, info_got)
        torch.cuda.synchronize()
        assert info_got.cpu().numpy().tolist() == [0] * batch
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        for b in range(batch):
            assert np.linalg.norm(g[b] - r[b]) / np.linalg.norm(r[b]) < 1e-12, (call, b)
            # and independently of the library: LAPACK's inverse of the same matrix
            want = np.linalg.inv(A[b])
            assert np.linalg.norm(g[b] - want) / np.linalg.norm(want) < 1e-11, (call, b)


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    import paper_2508_19138_gb300 as pkg
    n, batch = 416, 200
    need = pkg.bt_zinv_workspace_bytes(n, batch)
    assert need > (16 << 20)
    A = torch.zeros((batch, n, n), dtype=torch.complex128, device="cuda")
    info = torch.zeros(batch, dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.BTError) as ei:
        pkg.bt_zinv_batched_noalloc(n, A, n * n, batch, info)
    assert ei.value.status == pkg.BT_ERR_BUDGET
