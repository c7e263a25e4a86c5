"""C-ABI boundary checks that need no GPU: the library builds and loads, exports every entry
point declared in include/fuse.h, and its host-side validation answers correctly."""
import ctypes
import pathlib
import re

import pytest

from paper_2210_04184_gb300 import build, fuse

ROOT = pathlib.Path(__file__).resolve().parent.parent


def _declared():
    txt = (ROOT / "include" / "fuse.h").read_text()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fuse_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fuse.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "fuse_init" in names and "fuse_solve" in names and "fuse_weights" in names
    for name in names:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_has_same_names(lib):
    for name in _declared():
        assert callable(getattr(fuse, name)), name


def test_binding_constants_match_the_header():
    # every enumerator of include/fuse.h (statuses, dtypes, options, kernel groups) has the same
    # value in the Python binding
    txt = re.sub(r"/\*.*?\*/", "", (ROOT / "include" / "fuse.h").read_text(), flags=re.S)
    enums = re.findall(r"enum\s*(?:\w+\s*)?\{(.*?)\}", txt, flags=re.S)
    found = {}
    for body in enums:
        nxt = 0
        for item in (e.strip() for e in body.split(",")):
            if not item:
                continue
            m = re.fullmatch(r"(FUSE_\w+)\s*(?:=\s*(-?\d+))?", item)
            assert m, item
            nxt = int(m.group(2)) if m.group(2) is not None else nxt
            found[m.group(1)] = nxt
            nxt += 1
    assert "FUSE_OPT_X_UPDATE" in found and "FUSE_EUNSUPPORTED" in found
    for name, value in found.items():
        assert getattr(fuse, name) == value, name


def test_status_strings(lib):
    assert fuse.fuse_status_string(fuse.FUSE_OK) == "FUSE_OK"
    assert fuse.fuse_status_string(fuse.FUSE_EUNSUPPORTED) == "FUSE_EUNSUPPORTED"


def _ws(H=64, W=64, K=2, S=3, ratio=4, dtype=fuse.FUSE_F32, wdtype=fuse.FUSE_BF16, L=(93, 4, 20, 4)):
    g = fuse.fuse_geometry(H, W, L[0], L[1], L[2], L[3])
    return fuse.fuse_workspace_bytes(g, K, S, ratio, dtype, wdtype)


def test_workspace_bytes_counts_the_latent_state(lib):
    # Sigma dominates: (|W|/2) |P| L_s n_h elements in the default half-window mode
    # (24 * 25 * 20 * 256^2 * 4 B for the 256^2 case)
    b = _ws(H=256, W=256)
    sig = 24 * 25 * 20 * 256 * 256 * 4
    assert sig < b < sig * 1.1
    b64 = _ws(H=128, W=128, K=1, S=2, dtype=fuse.FUSE_F64, wdtype=fuse.FUSE_F64, L=(4, 1, 4, 1))
    assert b64 > 12 * 9 * 4 * 128 * 128 * 8


@pytest.mark.parametrize("kw,status", [
    (dict(H=70, W=64, ratio=2), fuse.FUSE_EUNSUPPORTED),  # 70 = 2*5*7: radix 7 unsupported
    (dict(H=64, W=66, ratio=2), fuse.FUSE_EUNSUPPORTED),  # W not a multiple of 4 for F32
    (dict(H=64, W=64, ratio=3), fuse.FUSE_EINVAL),        # H not divisible by the ratio
    (dict(K=4), fuse.FUSE_EUNSUPPORTED),                  # K > 3
    (dict(S=0), fuse.FUSE_EINVAL),
    (dict(H=8, W=8, K=2, S=2, ratio=1), fuse.FUSE_EINVAL),   # 2(K+S)+1 > 8
    (dict(dtype=fuse.FUSE_F64, wdtype=fuse.FUSE_BF16), fuse.FUSE_EUNSUPPORTED),
    (dict(dtype=fuse.FUSE_F32, wdtype=fuse.FUSE_F64), fuse.FUSE_EUNSUPPORTED),
])
def test_workspace_rejects_bad_geometry(lib, kw, status):
    with pytest.raises(fuse.FuseError) as e:
        _ws(**kw)
    assert e.value.status == status


def test_mixed_radix_sizes_accepted(lib):
    for n in (96, 120, 160, 192, 320, 384, 40):
        assert _ws(H=n, W=n, K=1, S=3) > 0
