"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
entry point include/pic.h declares, and the ctypes structures of the
binding have the C layout (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pic.h")


@pytest.fixture(scope="module")
def libpic():
    from paper_2206_14662_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(pic_[a-z_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(libpic):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(libpic, n), n


def test_strerror_without_gpu(libpic):
    libpic.pic_strerror.restype = ctypes.c_char_p
    assert libpic.pic_strerror(0) == b"ok"
    assert b"capacity" in libpic.pic_strerror(-3)


def test_binding_struct_layout(tmp_path):
    from paper_2206_14662_gb300 import _capi
    structs = {"pic_config": _capi.PicConfig, "pic_diag": _capi.PicDiag,
               "pic_kernel_times": _capi.PicKernelTimes, "pic_allocator": _capi.PicAllocator}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pic.h"', "int main(void){"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    for line in filter(None, out):
        cname, field, value = line.split()
        cls = structs[cname]
        got = ctypes.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert got == int(value), (cname, field)


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2206_14662_gb300 import _capi
    monkeypatch.setattr(_capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_capi, "_lib", None)
    with pytest.raises(RuntimeError):
        _capi.lib()


def test_batch_configurations_validated_on_the_host():
    """pic_init rejects, before touching a device, batches whose simulations
    disagree in the shared geometry or settings, and batch sizes outside
    1..256 (host logic; no GPU needed)."""
    from paper_2206_14662_gb300 import _capi
    from paper_2206_14662_gb300.inputs import scan_configs
    L = _capi.lib()
    h = ctypes.c_void_p()

    def init(cfgs, n=None):
        arr = (_capi.PicConfig * len(cfgs))(*[_capi.make_config(c) for c in cfgs])
        return L.pic_init(arr, len(cfgs) if n is None else n, None, None, ctypes.byref(h))

    base = scan_configs(n_sims=4, nr=32, nz=64, n_min=100, n_max=400)
    for field, value in (("nr", 33), ("r_out", 11e-3), ("dt", 2e-12), ("sort_every", 10),
                         ("precision", 64), ("seed", 2), ("poisson_rtol", 1e-9),
                         ("fixed_efield", 1)):
        bad = [dict(c) for c in base]
        bad[2][field] = value
        assert init(bad) == _capi.PIC_EINVAL, field
    assert init(base, n=0) == _capi.PIC_EINVAL
    assert init(base * 65, n=257) == _capi.PIC_EINVAL
    bad = [dict(c) for c in base]
    bad[3]["p_mbar"] = -1.0        # a per-simulation field is validated too
    assert init(bad) == _capi.PIC_EINVAL


def test_spline_and_trap_configurations_validated_on_the_host():
    """pic_init refuses, before touching a device, spline degrees outside
    0..3, a spline field with a seed source, a fixed field or a batch, and
    an ellipse without a spline degree or with a non-positive semi-axis."""
    from paper_2206_14662_gb300 import _capi
    from paper_2206_14662_gb300.inputs import workload
    L = _capi.lib()
    h = ctypes.c_void_p()

    def init(cfgs):
        arr = (_capi.PicConfig * len(cfgs))(*[_capi.make_config(c) for c in cfgs])
        return L.pic_init(arr, len(cfgs), None, None, ctypes.byref(h))

    base = workload("coax_32x64_1e4", precision=64)
    for deg in (-1, 4):
        assert init([dict(base, bspline_degree=deg)]) == _capi.PIC_EINVAL
    assert init([dict(base, bspline_degree=2, source_rate=1e9)]) == _capi.PIC_EINVAL
    assert init([dict(base, bspline_degree=2, fixed_efield=1)]) == _capi.PIC_EINVAL
    assert init([dict(base, bspline_degree=2)] * 2) == _capi.PIC_EINVAL
    ell = (9e-3, 0.0, 1e-3, 3e-3)
    assert init([dict(base, ellipse=ell)]) == _capi.PIC_EINVAL
    assert init([dict(base, bspline_degree=2, ellipse=(9e-3, 0.0, 0.0, 3e-3))]) == _capi.PIC_EINVAL
    # the binding sets the ellipse flag and axes
    c = _capi.make_config(dict(base, bspline_degree=2, ellipse=ell))
    assert c.has_ellipse == 1 and tuple(c.ellipse) == ell
