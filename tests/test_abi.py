"""The C-ABI library loads, exports every entry point include/bbdg.h declares, and rejects
bad input on the host (no GPU needed for these paths)."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from paper_1512_06025_gb300 import build as buildmod
from paper_1512_06025_gb300 import inputs


@pytest.fixture(scope="module")
def bb():
    buildmod.build()
    from paper_1512_06025_gb300 import bbdg
    bbdg.load()
    return bbdg


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(bbdg_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(bb):
    import ctypes
    lib = ctypes.CDLL(bb.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_num_nodes(bb):
    assert [bb.bbdg_num_nodes(N) for N in range(0, 12)] == [0, 4, 10, 20, 35, 56, 84, 120, 165, 220, 286, 0]


def test_rejects_inverted_element(bb):
    VX, EToV = inputs.kuhn_cube_mesh(1)
    E = EToV.copy()
    E[0, [2, 3]] = E[0, [3, 2]]
    K = len(E)
    with pytest.raises(bb.BBDGError) as ei:
        bb.bbdg_setup_mesh(VX, E, np.ones(K), np.ones(K))
    assert ei.value.code == -3 and "Jacobian" in str(ei.value)


def test_rejects_bad_materials_and_ids(bb):
    VX, EToV = inputs.kuhn_cube_mesh(1)
    K = len(EToV)
    with pytest.raises(bb.BBDGError) as ei:
        bb.bbdg_setup_mesh(VX, EToV, np.ones(K), -np.ones(K))
    assert ei.value.code == -1
    E = EToV.copy()
    E[1, 0] = 10_000
    with pytest.raises(bb.BBDGError) as ei:
        bb.bbdg_setup_mesh(VX, E, np.ones(K), np.ones(K))
    assert ei.value.code == -3


def test_rejects_non_manifold_face(bb):
    VX, EToV = inputs.kuhn_cube_mesh(1)
    E = np.concatenate([EToV, EToV[:1]])           # the same tetrahedron twice
    K = len(E)
    with pytest.raises(bb.BBDGError) as ei:
        bb.bbdg_setup_mesh(VX, E, np.ones(K), np.ones(K))
    assert ei.value.code == -3
