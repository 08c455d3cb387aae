"""The C-ABI library loads and exports every symbol include/mapdec.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os

import pytest

from paper_1802_08483_gb300 import build as libbuild
from paper_1802_08483_gb300 import mapdec


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return mapdec.load()


def test_header_symbols_exported(lib):
    syms = mapdec.header_symbols()
    assert "mapdec_create" in syms and "mapdec_decode" in syms and "mapdec_loglik_grad" in syms
    raw = ctypes.CDLL(mapdec.LIB_PATH)
    for s in syms:
        assert hasattr(raw, s), f"missing export {s}"
    # every exported entry point has a binding of the same name
    for s in syms:
        assert hasattr(mapdec, s), f"no python binding named {s}"


def test_strerror_names_every_status(lib):
    for st in range(8):
        assert mapdec.mapdec_strerror(st) != "unknown status"
    assert mapdec.mapdec_strerror(99) == "unknown status"


def test_header_documents_every_entry_point():
    import re
    txt = open(mapdec.HEADER).read()
    for s in mapdec.header_symbols():
        m = re.search(r"^[A-Za-z_][A-Za-z_0-9 ]*\**\s*\**" + s + r"\(", txt, flags=re.M)
        assert m, f"no declaration of {s}"
        before = txt[:m.start()].rstrip()
        assert before.endswith("*/"), f"{s} lacks a comment right above its declaration"


def test_library_does_not_link_oracle(lib):
    """The decoder library neither depends on the oracle's library nor imports or
    exports any oracle symbol: its dynamic section (NEEDED entries) and its
    dynamic symbol table, defined and undefined, are checked."""
    import shutil
    import subprocess
    readelf, nm = shutil.which("readelf"), shutil.which("nm")
    if not readelf or not nm:
        pytest.skip("binutils not available")
    dyn = subprocess.run([readelf, "-d", mapdec.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    needed = [ln for ln in dyn.splitlines() if "(NEEDED)" in ln]
    assert needed, "no NEEDED entries read"
    assert not any("oracle" in ln for ln in needed), needed
    syms = subprocess.run([nm, "-D", mapdec.LIB_PATH], capture_output=True, text=True,
                          check=True).stdout.split("\n")
    names = [ln.split()[-1] for ln in syms if ln.strip()]
    assert "mapdec_decode" in names
    assert not [s for s in names if s.startswith("orc_")], "oracle symbol in the library"


@pytest.mark.skipif(os.environ.get("CUDA_VISIBLE_DEVICES", None) is None and
                    __import__("torch").cuda.is_available(), reason="GPU present")
def test_no_gpu_fails_loudly(lib):
    """Without a usable device, create reports MAPDEC_ERR_CUDA (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import numpy as np
    cb = np.array([[0, 0], [1, 1]], np.uint8)
    with pytest.raises(mapdec.MapDecError) as e:
        mapdec.mapdec_create(2, 2, cb, 4, 0.01, 0.01, 0.0, 1, 4)
    assert e.value.status == mapdec.MAPDEC_ERR_CUDA


def test_constants_match_header():
    """Every status code and batch flag of the header has the same value in the
    binding (the binding restates them for ctypes callers)."""
    import re
    txt = re.sub(r"/\*.*?\*/", "", open(mapdec.HEADER).read(), flags=re.S)
    consts = dict((k, int(v)) for k, v in re.findall(r"\b(MAPDEC_[A-Z0-9_]+)\s*=\s*(\d+)", txt))
    assert "MAPDEC_BATCH_EXTRINSIC" in consts and "MAPDEC_ERR_ARG" in consts
    for k, v in consts.items():
        assert getattr(mapdec, k, None) == v, f"{k}: header {v}, binding {getattr(mapdec, k, None)}"
