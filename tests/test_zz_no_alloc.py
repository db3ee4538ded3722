"""The allocation-free demag product (mt_demag_field_noalloc).

Some callers cannot let the library allocate device memory (a loop that has
given all free HBM to cached tensors, code that cannot take the
synchronisation cudaMalloc may cause, or an application with its own pool).
For them the product runs with work areas from a fixed per-GPU array.  This
file checks, through the C ABI, that two calls in a row agree with the
allocating entry point within the FP32 field tolerance (1e-6), and that a
batch too large for the fixed array is refused.  It is collected last on
purpose.
"""
import numpy as np
import pytest

from paper_2107_05364_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2107_05364_gb300 import build
    build.build()
    from paper_2107_05364_gb300 import binding
    return binding


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_allocating_entry_twice(mt):
    import torch
    ctx = mt.mt_ctx_create(0)
    t = wl.graded_film(70, 19, 2, (350e-9, 95e-9, 6e-9), seed=12)  # n = 2660: ragged panels/chunks
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    B = 2
    for call, seed in enumerate((31, 47)):  # two calls in a row, different inputs
        m = np.stack([wl.m_random(t.n, seed=seed + b) for b in range(B)]).astype(np.float32)
        mg = torch.tensor(m.ravel(), device="cuda")
        H_ref = torch.full_like(mg, float("nan"))
        H = torch.full_like(mg, float("nan"))
        mt.mt_demag_field(T, mg, H_ref, B=B)
        mt.mt_demag_field_noalloc(T, mg, H, B=B)
        torch.cuda.synchronize()
        a, r = H.cpu().numpy(), H_ref.cpu().numpy()
        assert np.isfinite(a).all(), call
        assert _rel(a, r) <= 1e-6, (call, _rel(a, r))


def test_noalloc_refuses_batches_beyond_the_fixed_array(mt):
    import torch
    ctx = mt.mt_ctx_create(0)
    t = wl.film(60, 20, 1)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    B = 400  # about 6 MB of scaled operand: more than the 4 MiB array
    mg = torch.zeros(B * 3 * t.n, device="cuda")
    H = torch.zeros_like(mg)
    with pytest.raises(mt.MtError) as e:
        mt.mt_demag_field_noalloc(T, mg, H, B=B)
    assert e.value.status == mt.MT_EINVAL
    assert "MT_NOALLOC_SCRATCH_BYTES" in str(e.value)
