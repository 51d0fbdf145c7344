"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, exports
every function include/pf.h declares, validates arguments without a device,
and fails loudly (no CPU fallback) when no GPU is present."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(pf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    d = _declared()
    for n in ("pf_create", "pf_run", "pf_destroy", "pf_last_error", "pf_batch_run",
              "pf_server_create", "pf_server_submit", "pf_server_poll"):
        assert n in d


def test_library_exports_every_declared_symbol():
    import ctypes
    import paper_1306_3277_b300 as pf
    L = ctypes.CDLL(pf.library_path() if os.path.exists(pf.library_path()) else pf._build.build())
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_shape_queries_without_a_device():
    import paper_1306_3277_b300 as pf
    assert pf.pf_theta_size(pf.PF_WINDKESSEL) == 7
    assert pf.pf_theta_size(pf.PF_LORENZ96) == 5
    assert pf.pf_theta_size(9) == 0
    m = pf.model(pf.PF_LORENZ96, N=40, substeps=10, obs_stride=2, prec=pf.PF_MIXED)
    P, T = 1 << 20, 500
    b = pf.pf_device_bytes(m, P, T)
    assert b >= 2 * 40 * P * 4 + P * 8 + P * 4
    assert pf.pf_device_bytes(m, P, T, history=True) - b == T * P * 4
    assert pf.pf_device_bytes(pf.model(pf.PF_LORENZ96, N=7), 100, 10) == 0


def test_persistent_diagnostics_validate_without_a_device():
    """The persistent launch's test hooks refuse bad arguments on the host,
    before any CUDA call."""
    import paper_1306_3277_b300 as pf
    for bad in (0.0, -1.0, 60.5):
        with pytest.raises(pf.PFError) as e:
            pf.pf_debug_persist_wait_limit(bad)
        assert e.value.status == pf.PF_EINVAL
    assert pf.lib().pf_debug_persist_unfilled_slot(2) == pf.PF_EINVAL
    assert pf.lib().pf_debug_persist_unfilled_slot(-1) == pf.PF_EINVAL
    pf.pf_debug_persist_unfilled_slot(False)  # host-only: accepted without a device


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1306_3277_b300 as pf
    with pytest.raises(pf.PFError) as e:
        pf.pf_create(pf.model(pf.PF_WINDKESSEL), 1024, 100, 0.01)
    assert e.value.status == pf.PF_ECUDA


def test_product_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1306_3277_b300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, fn
                assert "pf_oracle" not in txt and "liboracle" not in txt, fn
