"""Checkpoint / resume of the integrator through the C ABI (no counterpart in
the paper): an image of the dynamic state (times, step sizes, step control,
counters, m and the first-same-as-last derivative of the Runge-Kutta (4,5)
step, Sec. 3.1) taken between calls and loaded into the same or another
integrator continues bit for bit, in fixed-step, adaptive and relax mode, on
the streaming and on the tensor-core (dense) product; damaged or mismatched
images are rejected and leave the integrator unchanged."""
import math

import numpy as np
import pytest

from paper_2107_05364_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MU0 = 4e-7 * math.pi
FIELD1 = np.array([-24.6e-3, 4.3e-3, 0.0]) / MU0


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
def ctx(mt):
    return mt.mt_ctx_create(0)


@pytest.fixture(scope="module")
def film(mt, ctx):
    t = wl.film(40, 10, 1)
    tiles = mt.mt_tiles_create(ctx, t)
    return t, tiles, mt.mt_demag_assemble(tiles, "f32")


def _batch(t, B, seed=0):
    return np.stack([wl.m_noisy(t.n, (1, 1, 1), 1e-2, seed=seed + b) for b in range(B)]).astype(np.float32)


def _params(mt, B):
    alpha = [0.02, 0.1, 0.5, 0.05][:B] + [0.02] * max(0, B - 4)
    Ha = np.tile(FIELD1, (B, 1)) * np.linspace(1.0, 0.5, B)[:, None]
    return mt.llg_params(B, alpha=alpha, Ha=Ha)


def _same_stats(a, b):
    for x, y in zip(a, b):
        for k in ("n_accept", "n_reject", "n_rhs", "t", "h", "tau", "status"):
            assert x[k] == y[k], (k, x[k], y[k])


def test_fixed_step_resume_is_bit_identical(mt, film, tmp_path):
    t, _, T = film
    B = 3
    p, keep = _params(mt, B)
    opts = mt.ode_opts(fixed_h=1e-13)
    I = mt.Integrator(T, p, opts, B)
    I.set_state(_batch(t, B).ravel())
    I.step(15)
    image = I.checkpoint()
    path = tmp_path / "ck.bin"
    path.write_bytes(image)  # a file round trip
    I.step(15)
    ya, sa = I.get_state(), I.stats()
    J = mt.Integrator(T, p, opts, B)
    J.restore(path.read_bytes())
    J.step(15)
    np.testing.assert_array_equal(J.get_state(), ya)
    _same_stats(J.stats(), sa)
    # back into the integrator that already went on
    I.restore(image)
    I.step(15)
    np.testing.assert_array_equal(I.get_state(), ya)


def test_image_before_first_step(mt, film):
    # taken right after set_state: the derivative is not evaluated yet, the
    # restored integrator evaluates it as the saved one would have
    t, _, T = film
    p, keep = _params(mt, 2)
    opts = mt.ode_opts(fixed_h=1e-13)
    I = mt.Integrator(T, p, opts, 2)
    I.set_state(_batch(t, 2, seed=5).ravel(), t0=1e-12)
    image = I.checkpoint()
    I.step(10)
    J = mt.Integrator(T, p, opts, 2)
    J.restore(image)
    J.step(10)
    np.testing.assert_array_equal(J.get_state(), I.get_state())
    _same_stats(J.stats(), I.stats())


def test_adaptive_resume_is_bit_identical(mt, film):
    t, _, T = film
    B = 3
    p, keep = _params(mt, B)
    opts = mt.ode_opts(rtol=1e-6, atol=1e-6)
    I = mt.Integrator(T, p, opts, B)
    I.set_state(_batch(t, B, seed=3).ravel())
    I.run(40e-12, 4)
    image = I.checkpoint()
    _, mavg_a, st_a = I.run(100e-12, 6)
    ya = I.get_state()
    J = mt.Integrator(T, p, opts, B)
    J.restore(image)
    _, mavg_b, st_b = J.run(100e-12, 6)
    np.testing.assert_array_equal(J.get_state(), ya)
    np.testing.assert_array_equal(mavg_b, mavg_a)
    _same_stats(st_b, st_a)
    assert all(s["n_accept"] > 0 for s in st_a)


def test_relax_resume_is_bit_identical(mt, film):
    t, _, T = film
    p, keep = mt.llg_params(2, alpha=[0.5, 0.5], Ha=np.zeros((2, 3)))
    opts = mt.ode_opts(rtol=1e-5, atol=1e-5)
    I = mt.Integrator(T, p, opts, 2)
    I.set_state(_batch(t, 2, seed=8).ravel())
    s, _ = I.relax(1e-4, 20e-12, check=False)  # stopped by the time cap
    assert s == mt.MT_ENOCONV
    image = I.checkpoint()
    s_a, st_a = I.relax(1e-4, 5e-9)
    J = mt.Integrator(T, p, opts, 2)
    J.restore(image)
    s_b, st_b = J.relax(1e-4, 5e-9)
    assert s_a == s_b == mt.MT_OK
    np.testing.assert_array_equal(J.get_state(), I.get_state())
    _same_stats(st_b, st_a)


def test_dense_tensor_core_resume(mt, ctx, film):
    t, tiles, _ = film
    T = mt.mt_demag_assemble_ex(tiles, "split", mt.MT_LAYOUT_DENSE)
    B = 8
    p, keep = _params(mt, B)
    opts = mt.ode_opts(rtol=1e-6, atol=1e-6)
    I = mt.Integrator(T, p, opts, B)
    I.set_state(_batch(t, B, seed=11).ravel())
    I.run(20e-12, 1)
    image = I.checkpoint()
    _, mavg_a, st_a = I.run(60e-12, 3)
    J = mt.Integrator(T, p, opts, B)
    J.restore(image)
    _, mavg_b, st_b = J.run(60e-12, 3)
    np.testing.assert_array_equal(J.get_state(), I.get_state())
    np.testing.assert_array_equal(mavg_b, mavg_a)
    _same_stats(st_b, st_a)


def test_restore_onto_other_precision(mt, film):
    # the saved derivative is dropped and re-evaluated on the BF16 tensor:
    # the continuation stays within the BF16 field tolerance of the FP32 one
    t, tiles, T = film
    Tb = mt.mt_demag_assemble(tiles, "bf16")
    p, keep = _params(mt, 1)
    opts = mt.ode_opts(fixed_h=1e-13)
    I = mt.Integrator(T, p, opts, 1)
    I.set_state(_batch(t, 1).ravel())
    I.step(10)
    image = I.checkpoint()
    I.step(10)
    J = mt.Integrator(Tb, p, opts, 1)
    J.restore(image)
    J.step(10)
    assert np.abs(J.get_state() - I.get_state()).max() <= 5e-3
    assert J.stats()[0]["t"] == I.stats()[0]["t"]


def test_bad_images_rejected(mt, film):
    t, _, T = film
    p, keep = _params(mt, 2)
    opts = mt.ode_opts(fixed_h=1e-13)
    I = mt.Integrator(T, p, opts, 2)
    I.set_state(_batch(t, 2).ravel())
    I.step(5)
    image = I.checkpoint()
    J = mt.Integrator(T, p, opts, 2)
    m_j = _batch(t, 2, seed=21)
    J.set_state(m_j.ravel())
    before = J.get_state()
    bad = bytearray(image)
    bad[len(bad) // 2] ^= 0x01  # one bit of m
    for img in (bytes(bad), image[:-1], image[:100], b"", b"NOTACKPT" + image[8:]):
        with pytest.raises(mt.MtError) as e:
            J.restore(img)
        assert e.value.status == mt.MT_EINVAL
    np.testing.assert_array_equal(J.get_state(), before)  # unchanged
    K = mt.Integrator(T, p, opts, 1)
    with pytest.raises(mt.MtError) as e:
        K.restore(image)  # B = 2 image into B = 1
    assert e.value.status == mt.MT_EINVAL


def test_image_moves_between_paths(mt, film):
    # an image taken on the one-kernel path continues on the step graph
    # to FP32 round-off of the product's summation order
    t, _, T = film
    p, keep = _params(mt, 2)
    opts = mt.ode_opts(fixed_h=1e-13)
    I = mt.Integrator(T, p, opts, 2)
    assert I.path() == mt.MT_PATH_PERSISTENT
    I.set_state(_batch(t, 2, seed=50).ravel())
    I.step(20)
    image = I.checkpoint()
    I.step(20)
    J = mt.Integrator(T, p, opts, 2)
    J.set_path(mt.MT_PATH_GRAPH)
    J.restore(image)
    J.step(20)
    assert np.abs(J.get_state() - I.get_state()).max() <= 1e-5
    for a, b in zip(J.stats(), I.stats()):
        for k in ("n_accept", "n_reject", "n_rhs", "status"):
            assert a[k] == b[k], (k, a[k], b[k])
        assert abs(a["t"] - b["t"]) <= 1e-9 * b["t"]
