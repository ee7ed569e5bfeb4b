"""CPU-side checks of the C ABI library: it builds for sm_103a, loads without a
GPU and exports every entry point that include/*.h declares; the binding
keeps the C names; host-side argument validation needs no device."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(ad_pic_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def cdll():
    from paper_2511_21839_gb300 import build
    from paper_2511_21839_gb300 import adpic

    build.build()
    return adpic.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["ad_pic_create", "ad_pic_set_lattice", "ad_pic_run", "ad_pic_moments", "ad_pic_set_beam",
              "ad_pic_destroy", "ad_pic_strerror", "ad_pic_save", "ad_pic_load"]:
        assert n in names


def test_library_exports_every_declared_symbol(cdll):
    for n in sorted(_declared()):
        assert hasattr(cdll, n), n


def test_binding_has_c_names():
    from paper_2511_21839_gb300 import adpic

    for n in _declared():
        assert hasattr(adpic, n), n


def test_strerror_and_kernel_names_need_no_gpu(cdll):
    from paper_2511_21839_gb300 import adpic

    assert adpic.ad_pic_strerror(0) == "ok"
    assert adpic.ad_pic_strerror(-6) == "particle outside the grid stencil"
    assert adpic.ad_pic_kernel_name(0) == "push"


@pytest.mark.parametrize("grid,N,P,prec", [((32, 32, 32), 100, 5, 0), ((32, 32, 32), 100, 7, 2), ((24, 32, 32), 100, 7, 0),
                                          ((4, 32, 32), 100, 7, 0), ((32, 32, 256), 100, 7, 0), ((32, 32, 32), 0, 7, 0)])
def test_create_rejects_bad_arguments_before_touching_the_device(cdll, grid, N, P, prec):
    from paper_2511_21839_gb300 import adpic

    with pytest.raises(adpic.AdPicError) as e:
        adpic.ad_pic_create(grid, N, P, prec)
    assert e.value.status == -1


def test_null_handle_is_invalid(cdll):
    assert cdll.ad_pic_run(None, 1) == -1
    assert cdll.ad_pic_set_lattice(None, None) == -1
