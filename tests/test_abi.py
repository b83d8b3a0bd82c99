"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/gsvr.h declares (no compute call is made here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points(header=None):
    """Entry points declared in include/*.h (or in one header)."""
    import glob
    names = set()
    for path in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        if header and os.path.basename(path) != header:
            continue
        src = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        names |= set(re.findall(r"\b(gsvr_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ["gsvr_create", "gsvr_destroy", "gsvr_set_stacks", "gsvr_set_observations",
                     "gsvr_set_gaussians", "gsvr_set_poses", "gsvr_forward", "gsvr_backward", "gsvr_adam_step"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2512_11624_b300.csrc import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2512_11624_b300 import cnn, gsvr
    assert sorted(gsvr.EXPORTS) == declared_entry_points("gsvr.h")
    assert sorted(cnn.EXPORTS) == declared_entry_points("gsvr_cnn.h")
    for n in gsvr.EXPORTS:
        assert callable(getattr(gsvr, n))
    for n in cnn.EXPORTS:
        assert callable(getattr(cnn.lib, n))
    assert gsvr.gsvr_abi_version() == 1


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        return
    from paper_2512_11624_b300 import gsvr
    try:
        gsvr.gsvr_create(0, stream=0)
    except gsvr.GsvrError as e:
        assert e.status == 1
    else:
        raise AssertionError("gsvr_create succeeded without a GPU")
