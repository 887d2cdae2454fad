"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol include/qmckl_gpu.h declares; host-side validation of the setters
runs without touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2512_16677_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qmckl_gpu.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2512_16677_gb300 import buildlib, qmckl
    buildlib.build()
    return qmckl.load()


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\bqk_status\s+(qk_\w+)\s*\(", txt)))


def test_header_symbols_exported(lib):
    names = _declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), f"{n} declared in the header but not exported"


def test_binding_covers_header():
    from paper_2512_16677_gb300 import qmckl
    assert set(_declared()) <= set(qmckl.SIGNATURES), \
        set(_declared()) - set(qmckl.SIGNATURES)


def _ctx():
    from paper_2512_16677_gb300 import qmckl
    return qmckl.Context("fp64")


def test_null_and_status_codes(lib):
    assert lib.qk_context_destroy(None) == -2
    assert lib.qk_set_precision(None, 53) == -2
    from paper_2512_16677_gb300 import qmckl
    c = _ctx()
    for bad in (1, 54):
        with pytest.raises(qmckl.QmcklError) as e:
            c.set_precision(bad)
        assert e.value.status == -1
    with pytest.raises(qmckl.QmcklError) as e:
        c.set_cutoff(0.0)
    assert e.value.status == -1
    with pytest.raises(qmckl.QmcklError) as e:
        c.lib.qk_set_compute_mode(c.h, 7) and c._check(c.lib.qk_set_compute_mode(c.h, 7), "m")
    assert e.value.status == -1


def test_setter_order_and_validation():
    from paper_2512_16677_gb300 import qmckl
    m = synth.make_config(1, walk_num=1)
    c = _ctx()
    with pytest.raises(qmckl.QmcklError) as e:      # basis before nuclei
        c.set_ao_basis(m.shell_nucleus, m.shell_ang_mom, m.shell_prim_num, m.shell_factor,
                       m.exponent, m.coefficient, m.prim_factor, m.ao_factor)
    assert e.value.status == -4
    c.set_nucleus(m.nucl_charge, m.nucl_coord)
    bad = m.nucl_coord.copy()
    bad[1, 2] = np.nan
    with pytest.raises(qmckl.QmcklError) as e:
        c.set_nucleus(m.nucl_charge, bad)
    assert e.value.status == -1
    with pytest.raises(qmckl.QmcklError) as e:      # MOs before basis
        c.set_mo_coefficient(m.mo_coef)
    assert e.value.status == -4

    def basis(**over):
        kw = dict(shell_nucleus=m.shell_nucleus, shell_ang_mom=m.shell_ang_mom,
                  shell_prim_num=m.shell_prim_num, shell_factor=m.shell_factor,
                  exponent=m.exponent, coefficient=m.coefficient, prim_factor=m.prim_factor,
                  ao_factor=m.ao_factor)
        kw.update(over)
        c.set_ao_basis(**kw)

    cases = [
        (dict(shell_nucleus=m.shell_nucleus + 5), -1),                  # nucleus out of range
        (dict(exponent=-m.exponent), -1),                               # gamma <= 0
        (dict(ao_factor=m.ao_factor[:-1]), -3),                         # ao_num mismatch
        (dict(shell_ang_mom=np.where(m.shell_ang_mom == 2, 4, m.shell_ang_mom)), -5),  # g shell
    ]
    for over, code in cases:
        with pytest.raises(qmckl.QmcklError) as e:
            basis(**over)
        assert e.value.status == code, (over.keys(), e.value)
    basis()
    assert c.ao_num == m.ao_num
    c.set_mo_coefficient(m.mo_coef)
    assert c.mo_num == m.mo_num
    with pytest.raises(qmckl.QmcklError) as e:      # nothing evaluated without points
        c.workspace_size()
    assert e.value.status == -4
    # empty point sets and unknown layouts are refused before any device call
    for pts, transp, code in ((np.zeros((0, 3)), "N", -3), (np.zeros((2, 0, 3)), "N", -3),
                              (np.zeros(0), "T", -3), (m.points[:4], "X", -1)):
        with pytest.raises(qmckl.QmcklError) as e:
            c.set_points(pts, transp=transp)
        assert e.value.status == code, (pts.shape, transp, e.value)
    assert c.lib.qk_set_points(c.h, b"N", 1, 4, None) == -2
    assert c.lib.qk_set_points_device(c.h, b"N", 1, 4, None) == -2
    c.close()


def test_last_error_truncates(lib):
    from paper_2512_16677_gb300 import qmckl
    c = _ctx()
    try:
        c.set_precision(99)
    except qmckl.QmcklError:
        pass
    buf = ctypes.create_string_buffer(8)
    assert lib.qk_last_error(c.h, buf, 8) == 0
    assert len(buf.value) == 7
    assert lib.qk_last_error(c.h, buf, 0) == -3


def test_missing_library_fails_loudly(tmp_path):
    """Without the built library the binding raises; nothing falls back to
    a CPU implementation."""
    import subprocess
    import sys
    code = ("from paper_2512_16677_gb300 import qmckl\n"
            f"qmckl.load({str(tmp_path / 'libqmckl_gpu.so')!r})\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode != 0
    assert "no CPU fallback" in r.stderr


class _FakeCuda:
    """Stands in for a CUDA tensor in the binding's checks (no GPU here)."""

    def __init__(self, dtype, n, contiguous=True):
        self.is_cuda, self.dtype, self._n, self._c = True, dtype, n, contiguous

    def is_contiguous(self):
        return self._c

    def numel(self):
        return self._n


def test_device_tensor_checks():
    """Tensors passed by pointer are checked before any CUDA call: device,
    layout, element type and, where the C call takes no size, the count."""
    torch = pytest.importorskip("torch")
    from paper_2512_16677_gb300 import qmckl
    chk = qmckl._device_tensor
    t = _FakeCuda(torch.float64, 12)
    assert chk(t, "x", torch.float64, numel=12, min_numel=12) is t
    bad = [(torch.zeros(4, 3, dtype=torch.float64), {}, "CUDA"),
           (_FakeCuda(torch.float64, 12, contiguous=False), {}, "contiguous"),
           (_FakeCuda(torch.float32, 12), {"dtype": torch.float64}, "dtype"),
           (_FakeCuda(torch.float64, 11), {"numel": 12}, "expected 12"),
           (_FakeCuda(torch.float64, 11), {"min_numel": 12}, "at least 12")]
    for x, kw, msg in bad:
        with pytest.raises(ValueError, match=msg):
            chk(x, "x", **kw)


def test_host_tensors_refused_before_any_device_call():
    torch = pytest.importorskip("torch")
    from paper_2512_16677_gb300 import qmckl
    m = synth.make_config(1, walk_num=1)
    c = _ctx()
    c.set_nucleus(m.nucl_charge, m.nucl_coord)
    c.set_ao_basis(m.shell_nucleus, m.shell_ang_mom, m.shell_prim_num, m.shell_factor,
                   m.exponent, m.coefficient, m.prim_factor, m.ao_factor)
    c.set_mo_coefficient(m.mo_coef)
    with pytest.raises(ValueError, match="CUDA"):
        c.set_points_device(torch.from_numpy(m.coord))
    with pytest.raises(ValueError, match="CUDA"):
        c.set_single_point_device(0, torch.zeros(1, 3, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA"):
        c.backward_device(torch.zeros(1, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA"):
        qmckl.contract_device(torch.zeros(2, 3), torch.zeros(4, 3))
    c.close()


def test_plain_c_consumer(lib, tmp_path):
    """The header compiles as C99 with warnings as errors, a C program links
    against the library and gets the documented status codes."""
    import shutil
    import subprocess
    from paper_2512_16677_gb300 import qmckl
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(qmckl.LIB_PATH)
    exe = tmp_path / "abi_consumer"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        f"-I{os.path.join(ROOT, 'include')}",
                        os.path.join(ROOT, "tests", "c", "abi_consumer.c"), "-o", str(exe),
                        f"-L{libdir}", "-lqmckl_gpu", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
