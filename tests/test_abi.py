"""The C-ABI library builds, loads without a GPU and exports every entry
point declared in include/mb.h and include/mb3.h (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header="mb.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(r"^\s*(?:mb_status|void|int|size_t|const char \*)\s*(mb3?_\w+)\s*\(", src, re.M)))


def test_header_declares_the_sweep_calls():
    names = declared()
    for n in ("mb_create", "mb_step", "mb_sweep", "mb_read_state", "mb_write_state", "mb_destroy"):
        assert n in names


@pytest.mark.parametrize("header", ["mb.h", "mb3.h"])
def test_library_exports_every_declared_symbol(header):
    from paper_1711_11361_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared(header)
    assert names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_every_export():
    from paper_1711_11361_gb300 import mb, mb3
    assert sorted(mb.EXPORTS) == declared("mb.h")
    assert sorted(mb3.EXPORTS) == declared("mb3.h")


def _noalloc_call(prob):
    """mb_cut_cells_noalloc on dummy output pointers: every case below fails
    its argument checks, which come before the first CUDA call, so no device
    is touched (and none is needed)."""
    import numpy as np
    from paper_1711_11361_gb300 import mb
    out = np.zeros(8)
    with pytest.raises(mb.MBError) as ei:
        mb.cut_cells_noalloc(prob, 0.0, 0.0, 0.0, out.ctypes.data, out.ctypes.data)
    return ei.value


def _square(n=4):
    import numpy as np
    t = np.linspace(0.0, 2.0 * np.pi, n, endpoint=False)
    return np.stack([0.5 + 0.2 * np.cos(t), 0.5 + 0.2 * np.sin(t)], axis=1)


def test_noalloc_rejects_too_many_vertices():
    from paper_1711_11361_gb300 import inputs, mb
    prob = inputs.Problem("many", 16, 16, 0.0, 0.0, 1.0, 1.0, polygons=[_square(16385)], moving=[1])
    e = _noalloc_call(prob)
    assert e.code == mb.MB_E_INVAL and "16384" in str(e)


def test_noalloc_rejects_degenerate_polygon():
    from paper_1711_11361_gb300 import inputs, mb
    prob = inputs.Problem("deg", 16, 16, 0.0, 0.0, 1.0, 1.0, polygons=[_square(2)], moving=[1])
    e = _noalloc_call(prob)
    assert e.code == mb.MB_E_INVAL and "fewer than 3" in str(e)


@pytest.mark.parametrize("x1,y1", [(0.0, 1.0), (1.0, 0.0), (-1.0, 1.0)])
def test_noalloc_rejects_empty_domain(x1, y1):
    from paper_1711_11361_gb300 import inputs, mb
    prob = inputs.Problem("empty", 16, 16, 0.0, 0.0, x1, y1, polygons=[_square(8)], moving=[1])
    e = _noalloc_call(prob)
    assert e.code == mb.MB_E_INVAL and "empty domain" in str(e)


# mb3_create checks every argument before its first CUDA call, so these
# run without a device: each must come back as MB_E_INVAL (-1)
def _mb3_invalid(**kw):
    import numpy as np
    from paper_1711_11361_gb300 import inputs, mb, mb3
    n, c, bb = inputs.cone_planes((0.5, 0.5, 0.5), 0.3, 0.2, 8)
    args = dict(normals=n, offsets=c, bbox=bb, U=(0.1, 0.0, 0.0))
    args.update(kw)
    dims = args.pop("dims", (8, 8, 8))
    p = inputs.Problem3("bad", *dims, **args)
    with pytest.raises(mb.MBError) as ei:
        mb3.Sim3(p, write_initial=False)
    return ei.value.code


@pytest.mark.parametrize("kw", [
    dict(dims=(1, 8, 8)),                                                   # one cell on an open axis
    dict(dims=(0, 8, 8)),
    dict(bc=(2, 0, 0, 0, 0, 0)),                                            # periodic on one side only
    dict(bc=(0, 0, 0, 0, 0, 3)),
    dict(gamma=1.0),
    dict(cfl=1.5),
    dict(cfl=0.0),
    dict(uncover_mode=5),
    dict(hi=(0.0, 1.0, 1.0)),                                               # hi <= lo
])
def test_mb3_create_rejects_bad_arguments(kw):
    assert _mb3_invalid(**kw) == -1


def test_mb3_create_rejects_too_many_planes():
    import numpy as np
    from paper_1711_11361_gb300 import inputs
    n, c, bb = inputs.cone_planes((0.5, 0.5, 0.5), 0.3, 0.2, 40)   # 41 planes > MB3_MAX_PLANES
    assert _mb3_invalid(normals=n, offsets=c, bbox=bb) == -1


def test_mb3_calls_reject_a_null_simulation():
    from paper_1711_11361_gb300 import mb3
    lib = mb3.lib
    assert lib.mb3_sweep(None, 0, 0.1) == -1
    assert lib.mb3_step(None, 0.1, None) == -1
    assert lib.mb3_set_precision(None, 1) == -1
    assert lib.mb3_flux_time(None, None) == -1
    assert lib.mb3_last_sweep(None, None, None) == -1
