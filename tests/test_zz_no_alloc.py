"""The allocation-free demag product (mt_demag_field_noalloc).

Some callers cannot let the library allocate device memory: a serving loop
that has handed all free HBM to cached tensors and must not fail half-way
through a step, code beside latency-critical streams that cannot take the
device-wide synchronisation cudaMalloc/cudaFree may cause, or an application
whose own memory pool forbids the CUDA allocator.  For them the product runs
with work areas from one fixed per-GPU array.  Through the C ABI this file
checks, for each streaming precision (FP32, scaled BF16, split BF16), on a
tensor that never saw the allocating entry point:
  - two calls in a row agree with the allocating entry point (run on a
    separately assembled copy of the tensor) within the field tolerance of
    that precision, and with the FP64 oracle's -N (Ms m) within the same
    tolerance (relative L2: FP32 and split 1e-6, BF16 5e-3);
  - after one warm-up call (which may load the kernels' device code), further
    calls leave the device's free memory unchanged: nothing is allocated;
  - a batch too large for the fixed array is refused.
It is collected last on purpose, and passes alone or after the other tests.
"""
import numpy as np
import pytest

import oracle
from paper_2107_05364_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-6, "bf16": 5e-3, "split": 1e-6}


@pytest.fixture(scope="module")
def mt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2107_05364_gb300 import build
    build.build()
    from paper_2107_05364_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def graded(mt):
    t = wl.graded_film(70, 19, 2, (350e-9, 95e-9, 6e-9), seed=12)  # n = 2660: ragged panels and chunks
    return t, oracle.Model.from_tiles(t)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["f32", "bf16", "split"])
def test_noalloc_matches_allocating_entry_and_oracle_twice(mt, graded, prec):
    import torch
    t, md = graded
    ctx = mt.mt_ctx_create(0)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, prec)      # only ever given to the no-alloc entry point
    T_ref = mt.mt_demag_assemble(tiles, prec)  # the allocating entry point's copy
    B = 2
    inputs = []
    for seed in (31, 47):
        m = np.stack([wl.m_random(t.n, seed=seed + b) for b in range(B)]).astype(np.float32)
        inputs.append((m, torch.tensor(m.ravel(), device="cuda")))
    H = torch.full_like(inputs[0][1], float("nan"))
    H_ref = torch.full_like(H, float("nan"))
    # warm-up: device code is loaded on first use, and the allocating entry
    # point makes its copy's work areas; from here on nothing may allocate
    mt.mt_demag_field_noalloc(T, inputs[0][1], H, B=B)
    mt.mt_demag_field(T_ref, inputs[0][1], H_ref, B=B)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call, (m, mg) in enumerate(inputs):  # two calls in a row, different inputs
        H.fill_(float("nan"))
        mt.mt_demag_field_noalloc(T, mg, H, B=B)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, (prec, call)
        mt.mt_demag_field(T_ref, mg, H_ref, B=B)
        torch.cuda.synchronize()
        a, r = H.cpu().numpy(), H_ref.cpu().numpy()
        assert np.isfinite(a).all(), (prec, call)
        assert _rel(a, r) <= TOL[prec], (prec, call, _rel(a, r))
        for b in range(B):
            ref = oracle.demag_field(md, m[b].astype(np.float64))
            got = a.reshape(B, t.n, 3)[b]
            assert _rel(got, ref) <= TOL[prec], (prec, call, b, _rel(got, ref))
    T.close()
    T_ref.close()
    tiles.close()


def test_noalloc_refuses_batches_beyond_the_fixed_array(mt):
    import torch
    ctx = mt.mt_ctx_create(0)
    t = wl.film(60, 20, 1)
    tiles = mt.mt_tiles_create(ctx, t)
    T = mt.mt_demag_assemble(tiles, "f32")
    B = 400  # 480,000 tile-simulations: about 6.7 MB of scratch, more than the 4 MiB array
    mg = torch.zeros(B * 3 * t.n, device="cuda")
    H = torch.zeros_like(mg)
    with pytest.raises(mt.MtError) as e:
        mt.mt_demag_field_noalloc(T, mg, H, B=B)
    assert e.value.status == mt.MT_EINVAL
    assert "MT_NOALLOC_SCRATCH_BYTES" in str(e.value)
