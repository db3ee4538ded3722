"""CPU-side checks of the boundary: the library builds for sm_103a, loads
without a GPU, and exports every entry point include/mt.h declares; the
host logic of the stream-K split is consistent."""
import ctypes
import os
import re

import numpy as np

from paper_2107_05364_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mt.h")).read()
    return sorted(set(re.findall(r"^MT_API\s+[\w\s\*]*?\b(mt_\w+)\s*\(", src, flags=re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    names = _declared()
    assert len(names) >= 20, names
    L = ctypes.CDLL(path)
    for name in names:
        assert hasattr(L, name), name
    from paper_2107_05364_gb300 import binding
    assert set(binding.exported_symbols()) <= set(names)
    missing = set(names) - set(binding.exported_symbols())
    assert not missing, "binding lacks %s" % sorted(missing)
    assert binding.mt_version().startswith("magtile")


def test_no_device_is_reported_cleanly():
    # without a GPU the context call fails with a status, not a crash
    import torch
    if torch.cuda.is_available():
        return
    from paper_2107_05364_gb300 import binding
    try:
        binding.mt_ctx_create(0)
    except binding.MtError as e:
        assert e.status in (binding.MT_EINVAL, binding.MT_ECUDA)
    else:
        raise AssertionError("context creation without a GPU must fail")


def _sk_begin(k, U, G):
    return (k * U) // G


def _sk_owner(u, U, G):
    return ((u + 1) * G + U - 1) // U - 1


def test_stream_k_split_covers_units_once():
    # the split used by the streaming product: CTA k owns [begin(k), begin(k+1));
    # owner(u) must be the CTA whose range holds u, for every u, including
    # the case of fewer units than CTAs
    rng = np.random.default_rng(0)
    for U, G in [(1, 152), (7, 152), (152, 152), (153, 152), (49375, 152), (1000, 7)] + \
            [(int(rng.integers(1, 5000)), int(rng.integers(1, 300))) for _ in range(30)]:
        owners = np.array([_sk_owner(u, U, G) for u in range(U)])
        for u in range(U):
            k = owners[u]
            assert _sk_begin(k, U, G) <= u < _sk_begin(k + 1, U, G), (U, G, u, k)
        assert _sk_begin(G, U, G) == U and _sk_begin(0, U, G) == 0


def test_sources_name_no_closed_calls():
    # batched async memcpy entry points are not used anywhere in the sources
    bad = re.compile(r"Memcpy(3D)?BatchAsync")
    for d in ("paper_2107_05364_gb300", "include", "oracle"):
        for dp, _, fs in os.walk(os.path.join(ROOT, d)):
            for f in fs:
                if f.endswith((".cu", ".cuh", ".h", ".c", ".py")):
                    assert not bad.search(open(os.path.join(dp, f)).read()), f


def test_binding_refuses_host_and_malformed_buffers():
    # The product entry points take raw device pointers of B * 3n elements;
    # the binding refuses anything else before calling the library (a host
    # array or a short buffer would otherwise become an out-of-bounds device
    # access).  No GPU is needed: the checks run first.
    import types

    import pytest
    import torch

    from paper_2107_05364_gb300 import binding as mt
    n = 10
    T = types.SimpleNamespace(n=n, h=None, tiles=types.SimpleNamespace(ctx=types.SimpleNamespace(device=0)))
    good_host = np.zeros(3 * n, np.float32)
    cpu_t = torch.zeros(3 * n)
    for f in (mt.mt_demag_field, mt.mt_demag_field_noalloc):
        with pytest.raises(ValueError, match="torch CUDA tensor"):
            f(T, good_host, good_host)
        with pytest.raises(ValueError, match="host memory"):
            f(T, cpu_t, cpu_t)
        with pytest.raises(ValueError, match="B must be"):
            f(T, cpu_t, cpu_t, B=0)
    with pytest.raises(ValueError, match="host memory"):
        mt.mt_demag_field_f64(T, cpu_t.double(), cpu_t.double())
    p, keep = mt.llg_params(1)
    with pytest.raises(ValueError, match="host memory"):
        mt.mt_llg_rhs(T, p, cpu_t, cpu_t)
    with pytest.raises(ValueError, match="host memory"):
        mt.mt_energy(T, p, cpu_t)
    with pytest.raises(ValueError, match="host memory"):
        mt.mt_relax(T, p, mt.ode_opts(), cpu_t, 1e-4, 1e-9)
    with pytest.raises(ValueError, match="host memory"):
        mt.mt_integrate(T, p, mt.ode_opts(), cpu_t, 0.0, 1e-9)
