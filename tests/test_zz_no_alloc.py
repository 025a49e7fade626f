"""fhe_rescale_noalloc: the rescale entry point for callers that cannot allocate device
memory (it takes its scratch from a fixed array inside the library instead of from the
caller or from cudaMalloc). Its output must equal fhe_rescale's, bit for bit, call after
call: the shared array keeps the previous call's contents, which must not leak into the next
result. The calls alternate between a large and a small shape, so each call runs over
leftovers of a different layout, and the reference runs use scratch filled with all-ones
words, so a read of a scratch word that the rescale did not write first would differ from
the reference. Collected last on purpose."""
import numpy as np
import pytest

from oracle import params as P
from paper_2212_14191_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fhe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_14191_gb300 import fhe as f
    return f


def test_noalloc_rescale_matches_rescale(fhe):
    import torch
    qs, ps = P.default_moduli(24, 8)
    ctx = fhe.Context(16, qs, ps, alpha=8)
    stream = torch.cuda.current_stream().cuda_stream
    for call, (logn, nl, batch) in enumerate([(16, 24, 2), (12, 5, 3), (16, 24, 2), (14, 9, 1)]):
        n = 1 << logn
        need = fhe.fhe_scratch_bytes(ctx.handle, fhe.FHE_OP_RESCALE, logn, nl, batch)
        assert 0 < need <= fhe.FHE_RESCALE_NOALLOC_MAX_BYTES
        scratch = torch.full((need // 4,), -1, dtype=torch.int32, device="cuda")
        x = I.uniform_residues(300 + call, qs[:nl], 2 * batch, n)
        ct = fhe.to_device(x.reshape(nl, 2, batch, n).transpose(1, 0, 2, 3).copy())
        want = torch.empty((2, nl - 1, batch, n), dtype=torch.int32, device="cuda")
        got = torch.full_like(want, -1)
        fhe.fhe_rescale(ctx.handle, logn, nl, batch, ct.data_ptr(), want.data_ptr(), scratch.data_ptr(),
                        need, stream)
        fhe.fhe_rescale_noalloc(ctx.handle, logn, nl, batch, ct.data_ptr(), got.data_ptr(), stream)
        torch.cuda.synchronize()
        assert torch.equal(got, want), (call, logn, nl, batch)
    ctx.close()


def test_noalloc_rejects_oversize(fhe):
    import torch
    qs, ps = P.default_moduli(24, 8)
    ctx = fhe.Context(16, qs, ps, alpha=8)
    nl, batch = 24, 64   # 48 limbs x 64 x 2^16 x 4 B = 768 MiB of scratch > the fixed array
    assert fhe.fhe_scratch_bytes(ctx.handle, fhe.FHE_OP_RESCALE, 16, nl, batch) > fhe.FHE_RESCALE_NOALLOC_MAX_BYTES
    d = torch.zeros(16, dtype=torch.int32, device="cuda")
    with pytest.raises(fhe.FheError) as e:
        fhe.fhe_rescale_noalloc(ctx.handle, 16, nl, batch, d.data_ptr(), d.data_ptr(), 0)
    assert e.value.code == fhe.FHE_ENOMEM and "FHE_RESCALE_NOALLOC_MAX_BYTES" in str(e.value)
    ctx.close()
