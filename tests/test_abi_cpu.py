"""C-ABI checks that need no GPU: the library loads, exports every entry point the
header declares, validates descriptors, and its host planner produces exactly the
oracle's level structure (greedy colours, merged near/fill block CSR and kinds)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import structure as st

from conftest import ROOT, problem

HEADER = os.path.join(ROOT, "include", "h2rs.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"H2_API\s+[\w\s\*]+?\b(h2_\w+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    from paper_2509_11152_b300 import binding
    lib = binding.lib()
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTED) == names
    assert binding.h2_version().startswith("h2rs")


def _oracle_levels(A):
    """Oracle structure of every skeletonised level (leaves first)."""
    t = A.top_level()
    out = []
    carried = set()
    for l in range(A.depth, t - 1, -1):
        nbrs = st.neighbours(A, l)
        fill = st.fill_pattern(nbrs, carried)
        lay = st.level_layout(nbrs, fill, [1] * len(nbrs))
        out.append((st.greedy_colouring(nbrs), lay))
        pn = st.neighbours(A, l - 1)
        pnear = {(p, q) for p in range(len(pn)) for q in pn[p]}
        carried = st.carried_to_parent(fill, pnear)
    return out


@pytest.mark.parametrize("name,over", [
    ("cov2d", dict(n=1024, leaf=32)),
    ("cov2d", {}),
    ("laplace2d", dict(n=4096, leaf=32, eta=0.7)),
    ("matern3d", dict(n=2048, leaf=32)),
    ("sphere", dict(n=8192, leaf=64)),
    ("gauss3d", dict(n=1500, leaf=32)),
])
def test_plan_matches_oracle_structure(name, over):
    from paper_2509_11152_b300 import h2_plan_query
    A = problem(name, **over).A
    for li, (colour, lay) in enumerate(_oracle_levels(A)):
        q = h2_plan_query(A, li)
        assert np.array_equal(q["colour"], np.asarray(colour, np.int32))
        assert np.array_equal(q["row_ptr"], lay["row_ptr"])
        assert np.array_equal(q["col"], lay["col"])
        assert np.array_equal(q["kind"], lay["kind"].astype(np.int32))


def test_descriptor_validation_errors():
    from paper_2509_11152_b300 import binding
    A = problem("cov2d", n=512, leaf=32).A
    d, keep = binding.make_desc(A)
    nbox = ctypes.c_int64()
    rc = binding.lib().h2_plan_query(ctypes.byref(d), 0, ctypes.byref(nbox), None, None, None, None, None)
    assert rc == 0 and nbox.value == 16
    # a child range that does not partition its parent
    bad = keep["node_size"].copy()
    bad[1] += 1
    d.node_size = bad.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    rc = binding.lib().h2_plan_query(ctypes.byref(d), 0, None, None, None, None, None, None)
    assert rc == -1 and b"partition" in binding.lib().h2_last_error()
    d.node_size = keep["node_size"].ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    # a level out of range
    rc = binding.lib().h2_plan_query(ctypes.byref(d), 99, None, None, None, None, None, None)
    assert rc == -1
    # a null descriptor
    rc = binding.lib().h2_plan_query(None, 0, None, None, None, None, None, None)
    assert rc == -1
