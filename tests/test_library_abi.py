"""The C-ABI library builds, loads and exports every symbol include/lightfuse.h
declares (no GPU needed: only host-side calls are made)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lightfuse.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lf_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2608_29269_b300.build import build
    from paper_2608_29269_b300 import _native
    build()
    return _native.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_declares_every_symbol():
    from paper_2608_29269_b300 import _native
    assert sorted(s[0] for s in _native.SIGNATURES) == declared_functions()


def test_host_only_calls(lib):
    from paper_2608_29269_b300 import _native as N
    p = N.LfParams()
    assert lib.lf_params_default(C.byref(p)) == 0
    assert abs(p.alpha_max - 0.99) < 1e-7 and p.max_rounds == 64
    assert lib.lf_params_default(None) == N.LF_ERR_INVALID
    assert lib.lf_shade_scratch_bytes(800, 800, 16) >= 28 * 4 * 800 * 800 * 16
    assert lib.lf_backward_scratch_bytes(800, 800, 16) >= 9 * 4 * 800 * 800 + lib.lf_shade_scratch_bytes(800, 800, 16)
    assert lib.lf_backward_scratch_bytes(0, 5, 4) == 0 and lib.lf_shade_scratch_bytes(8, 8, 0) == 0
    assert lib.lf_create(C.byref(p), None, None) == N.LF_ERR_INVALID
    bad = N.LfParams()
    lib.lf_params_default(C.byref(bad))
    bad.alpha_max = 1.5
    h = C.c_void_p()
    assert lib.lf_create(C.byref(bad), None, C.byref(h)) == N.LF_ERR_INVALID
    assert lib.lf_sync(None) == N.LF_ERR_INVALID
    assert lib.lf_destroy(None) == N.LF_ERR_INVALID
    assert lib.lf_last_error(None) == b"null context"


def test_params_agree_with_oracle_readings(lib):
    """Both sides state the same readings of the paper's open constants."""
    import oracle
    from paper_2608_29269_b300 import _native as N
    p = N.LfParams()
    lib.lf_params_default(C.byref(p))
    o = oracle.default_params()
    for k in ["T_min", "alpha_min", "alpha_max", "support_r2", "eps_w", "t_min", "ray_offset", "p_spec"]:
        assert abs(getattr(p, k) - o[k]) <= 1e-7 * max(1.0, abs(o[k])), k


def test_product_path_fails_loudly_without_extension(tmp_path):
    from paper_2608_29269_b300 import _native
    saved = _native._lib
    _native._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            _native.load(str(tmp_path / "missing.so"))
    finally:
        _native._lib = saved


def test_gbuffer_channels_agree_with_header():
    """The binding's G-buffer plane indices and count are the header's enum."""
    from paper_2608_29269_b300 import _native as N
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    enum = {k: int(v) for k, v in re.findall(r"\b(LF_CH_[A-Z_]+|LF_GBUF_[A-Z]+)\s*=\s*(\d+)", text)}
    assert enum["LF_GBUF_CHANNELS"] == N.LF_GBUF_CHANNELS
    assert enum["LF_GBUF_DIFF"] == N.LF_GBUF_DIFF
    names = dict(T="LF_CH_T", W="LF_CH_W", depth="LF_CH_DEPTH", x="LF_CH_X", n="LF_CH_N", a="LF_CH_A",
                 m="LF_CH_M", r="LF_CH_R", rho="LF_CH_RHO", nlen="LF_CH_NLEN", hits="LF_CH_HITS",
                 t_stop="LF_CH_TSTOP", id_stop="LF_CH_IDSTOP", dir="LF_CH_DIR", stopkey_lo="LF_CH_STOPKEY_LO",
                 x_lo="LF_CH_X_LO", n_lo="LF_CH_N_LO", r_lo="LF_CH_R_LO")
    assert set(names) == set(N.CH)
    for k, h in names.items():
        assert N.CH[k] == enum[h], k
    # planes are disjoint and fill the buffer
    width = dict(x=3, n=3, a=3, rho=3, dir=3, x_lo=3, n_lo=3)
    used = sorted(c for k, c0 in N.CH.items() for c in range(c0, c0 + width.get(k, 1)))
    assert used == list(range(N.LF_GBUF_CHANNELS))
